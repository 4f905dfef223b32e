"""CPU model of the digit GEMM's pre-tiled plane layout (gemm_oz.cu).

The split kernels write value (b, r, k) of slice s at BF16 index
    ((((b G + r/8) KB + k/16) ns + s) 2 + (k/8) % 2) 64 + (r % 8) 8 + k % 8
(G = ceil(rows / 8), KB = Kp / 16).  This model replays, in the kernels' own index
arithmetic, (1) the row-major writer (a warp per 8-row group and K segment, lane =
4 (r % 8) + j, two k per lane), (2) the transposing writer (32 x 64 tiles through shared
memory) and (3) the reads of one pipeline stage: the 5-d TMA box {256-byte run, slice,
K block, row group, batch} landing as [group][slice][256 B], then the MMA descriptors'
core-matrix walk (leading offset 128 bytes between the two K halves, stride offset
ns x 256 bytes between 8-row groups, slice tiles 256 bytes apart).  It checks that every
plane element is written exactly once and inside the allocation, that every stage read
stays inside the stage, and that the descriptor walk reads exactly op(X)[r][k] of the
slice (or a zero-filled row beyond the last group).
"""
import pytest


def layout(b, r, k, s, G, KB, ns):
    return ((((b * G + r // 8) * KB + k // 16) * ns + s) * 2 + (k // 8) % 2) * 64 + (r % 8) * 8 + k % 8


def check(rows, K, batch, ns, box_rows=128, seg=1024):
    Kp = max(64, (K + 63) // 64 * 64)
    G, KB = (rows + 7) // 8, Kp // 16
    total = ns * batch * G * 8 * Kp
    # rows writer
    seen = {}
    nseg = (Kp + seg - 1) // seg
    for item in range(batch * G * nseg):
        bg, sg = divmod(item, nseg); b, g = divmod(bg, G)
        h0, h1 = sg * (seg // 8), min(Kp, (sg + 1) * seg) // 8
        assert (h1 - h0) % 4 == 0
        for lane in range(32):
            r = g * 8 + (lane >> 2)
            for hb in range(h0, h1):
                kb = hb >> 1; h = hb & 1
                for t in range(2):
                    k = hb * 8 + (lane & 3) * 2 + t
                    base = ((bg * KB + kb) * ns) * 128
                    for s in range(ns):
                        idx = base + s * 128 + h * 64 + (lane >> 2) * 8 + (lane & 3) * 2 + t
                        assert 0 <= idx < total
                        assert idx == layout(b, r, k, s, G, KB, ns), (b, r, k, s)
                        assert idx not in seen; seen[idx] = (b, r, k, s)
    assert len(seen) == total
    # cols writer
    seen2 = set()
    rt, kt = (G + 3) // 4, Kp // 64
    for t in range(rt * kt * batch):
        b, rem = divmod(t, rt * kt); r0 = (rem // kt) * 32; k0 = (rem % kt) * 64
        for ty in range(8):
            for tx in range(32):
                rr, jj = tx >> 2, tx & 3
                for c in range(ty, 32, 8):
                    gl, hl = c >> 3, c & 7
                    g = (r0 >> 3) + gl
                    if g >= G: continue
                    r = g * 8 + rr
                    kl = hl * 8 + jj * 2
                    kb = (k0 >> 4) + (hl >> 1)
                    base = (((b * G + g) * KB + kb) * ns) * 128
                    for u in range(2):
                        # tile[kl + u][gl*8 + rr] holds X[k0 + kl + u][r0 + gl*8 + rr]
                        assert r0 + gl * 8 + rr == r
                        k = k0 + kl + u
                        for s in range(ns):
                            idx = base + s * 128 + (hl & 1) * 64 + rr * 8 + jj * 2 + u
                            assert idx == layout(b, r, k, s, G, KB, ns)
                            assert idx not in seen2; seen2.add(idx)
    assert len(seen2) == total
    # TMA box + descriptor reads
    ntile = (rows + box_rows - 1) // box_rows
    stage_bytes = ns * box_rows * 16 * 2
    for b in range(batch):
        for mt in range(ntile):
            for kb in range(KB):
                g0 = mt * box_rows // 8
                smem = {}
                for gl in range(box_rows // 8):
                    for s in range(ns):
                        for x in range(128):
                            off = (gl * ns + s) * 256 + 2 * x
                            assert off + 2 <= stage_bytes
                            g = g0 + gl
                            smem[off] = None if g >= G else ((((b * G + g) * KB + kb) * ns + s) * 128 + x)
                LBO, SBO = 128, ns * 256
                for s in range(ns):
                    for m in range(box_rows):
                        for kk in range(16):
                            off = s * 256 + (m // 8) * SBO + (kk // 8) * LBO + (m % 8) * 16 + (kk % 8) * 2
                            v = smem[off]
                            r = mt * box_rows + m
                            if v is None:
                                assert r // 8 >= G
                            else:
                                assert v == layout(b, r, kb * 16 + kk, s, G, KB, ns)
    return True


@pytest.mark.parametrize("rows,K,batch,ns", [(13, 70, 2, 5), (128, 64, 1, 5), (200, 130, 1, 7),
                                             (48, 2000, 1, 7), (9, 64, 3, 3)])
def test_layout_writers_and_stage_reads_agree(rows, K, batch, ns):
    assert check(rows, K, batch, ns)


def test_half_tiles_of_the_seven_digit_form():
    assert check(200, 130, 1, 7, box_rows=64)     # 128 x 64 tiles: B boxes of 8 groups


def test_segmented_row_writer():
    assert check(70, 1100, 1, 4, seg=1024)
