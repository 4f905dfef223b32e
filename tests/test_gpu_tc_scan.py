"""Transition-point search on the GPU (Gu-Wen ratio X of batched instances, Sec. III D):
every evaluated X equals the oracle's X for the same coupling (FP64 form, same
sketches), and the search keeps the interval where X crosses 1.5."""
import numpy as np
import pytest

from oracle import trg_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trg(require_gpu):
    import paper_2507_21909_b300 as pkg
    return pkg


def test_tc_scan_matches_oracle(trg):
    from paper_2507_21909_b300.tc_scan import tc_scan
    D, nsteps = 5, 12
    res = tc_scan(0.13, 0.17, D=D, nsteps=nsteps, points=5, rounds=1, lanes=3, precision=0)
    betas, X = res["history"][0]
    for b, x in zip(betas, X):
        st = O.init_ising(4, float(b), 0.0)
        for n in range(nsteps):
            O.step(st, n % 4, D, 2 * D, 4, 4, 0x5EED)
            dg = st.diag[-1]
            assert min([dg["gap_swap"]] + list(dg["gap_sq"].values())) > 1e-4, (b, n)
        assert abs(x - O.gu_wen_ratio(st)) < 1e-9, (b, x)
    assert res["interval"] == pytest.approx((0.14, 0.15))
    assert 0.14 <= res["beta_c"] <= 0.15
    assert res["T_c"] == pytest.approx(1.0 / res["beta_c"])
