"""Host logic of the per-step JSON-lines log, on a stand-in for the binding."""
import math

from paper_2507_21909_b300.steplog import StepLog, read_log


class FakeLib:
    def __init__(self):
        self.n = 0
        self.calls = []

    def trg_step(self, axis, D, p):
        self.calls.append((axis, D, p))
        self.n += 1

    def trg_diag(self):
        return -0.5 * self.n, (math.inf if self.n == 1 else 0.01 * self.n), self.n

    def trg_state_dims(self, which=0):
        return (4, 4, 4, 4, 4)

    def trg_step_timings(self):
        return {"resplit": 1.0, "norm": 0.1}

    def trg_free_energy(self):
        return -4.9 - self.n, 0.7 + self.n


def test_steplog_records_each_step(tmp_path):
    path = tmp_path / "run.jsonl"
    lib = FakeLib()
    with StepLog(str(path), lib=lib) as log:
        for n in range(3):
            log.step(n % 4, 4, 8)
    recs = read_log(str(path))
    assert [r["step"] for r in recs] == [1, 2, 3]
    assert [r["axis"] for r in recs] == [0, 1, 2]
    assert recs[0]["min_gap"] is None and recs[1]["min_gap"] == 0.02
    assert recs[2]["log_c"] == -1.5 and recs[2]["lnZ_per_site"] == 3.7
    assert recs[0]["dims"] == [4, 4, 4, 4, 4] and recs[0]["phases_ms"]["resplit"] == 1.0
    assert lib.calls == [(0, 4, 8), (1, 4, 8), (2, 4, 8)]


def test_steplog_appends_and_skips_free_energy(tmp_path):
    path = tmp_path / "run.jsonl"
    for _ in range(2):
        with StepLog(str(path), lib=FakeLib(), with_free_energy=False) as log:
            log.step(3, 6, 12)
    recs = read_log(str(path))
    assert len(recs) == 2 and all("f" not in r for r in recs)
