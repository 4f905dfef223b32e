"""Per-step JSON-lines log of a coarse-graining run (host side).

After each step it appends one line: the step index, axis, D and p, ln c_n, the
smallest relative gap at the step's cuts (bond swap and squeezers; a small gap flags a
near-degenerate truncation), the coarse tensor's shape, the per-phase device times,
and, if requested, ln Z/V so far.  Everything is read through the library's own calls
(trg_diag, trg_state_dims, trg_step_timings, trg_free_energy); `lib` is the binding
module, or any object with those functions.
"""
from __future__ import annotations

import json
import time


class StepLog:
    def __init__(self, path: str, lib=None, with_free_energy: bool = True):
        if lib is None:
            from . import _lib as lib
        self.lib = lib
        self.path = path
        self.with_free_energy = with_free_energy
        self._f = open(path, "a", encoding="utf-8")

    def step(self, axis: int, D: int, p: int) -> dict:
        """Run one trg_step and log it; returns the logged record."""
        t0 = time.perf_counter()
        self.lib.trg_step(axis, D, p)
        wall = time.perf_counter() - t0
        log_c, gap, nsteps = self.lib.trg_diag()
        rec = {"step": nsteps, "axis": axis, "D": D, "p": p, "log_c": log_c,
               "min_gap": gap if gap == gap and gap != float("inf") else None,
               "dims": list(self.lib.trg_state_dims()), "wall_s": wall,
               "phases_ms": self.lib.trg_step_timings()}
        if self.with_free_energy:
            rec["f"], rec["lnZ_per_site"] = self.lib.trg_free_energy()
        self._f.write(json.dumps(rec) + "\n")
        self._f.flush()
        return rec

    def close(self):
        self._f.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def read_log(path: str) -> list[dict]:
    with open(path, encoding="utf-8") as f:
        return [json.loads(line) for line in f if line.strip()]
