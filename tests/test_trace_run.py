"""The per-run analysis trace (host logic, CPU only): rows at every interval,
the mass drift against the first row, JSON lines on disk, and the early stop
on an unstable state, driven by a stand-in for a Domain."""
import json

import pytest

import paper_2007_12266_gb300 as lbm


class _Sim:
    """A stand-in with the Domain calls trace_run uses."""

    def __init__(self, unstable_at=None):
        self.step = 0
        self.unstable_at = unstable_at
        self.advanced = []

    def advance(self, n):
        self.advanced.append(n)
        self.step += n

    def measure(self):
        s = self.step
        return {"step": s, "sat_mass": 0.4 + 1e-4 * s, "sat_count": 0.41, "flux": [0.0, 0.0, 1e-5 * s],
                "flux_a": [0.0, 0.0, 4e-6 * s], "flux_b": [0.0, 0.0, 6e-6 * s], "ca": 1e-4,
                "mass_a": 400.0 + 0.001 * s, "mass_b": 600.0, "status": 1 if self.unstable_at == s else 0}


def test_rows_at_every_interval_and_on_disk(tmp_path):
    sim = _Sim()
    path = tmp_path / "trace.jsonl"
    rows = lbm.trace_run(sim, 250, 100, str(path))
    assert sim.advanced == [100, 100, 50]                  # the last chunk is the remainder
    assert [r["step"] for r in rows] == [0, 100, 200, 250]
    assert set(rows[0]) == set(lbm.TRACE_FIELDS)
    assert rows[0]["mass_drift"] == 0.0
    assert rows[-1]["mass_drift"] == pytest.approx(0.25 / 1000.0, rel=1e-12)
    assert rows[-1]["flux"][2] == pytest.approx(2.5e-3)
    on_disk = [json.loads(l) for l in path.read_text().splitlines()]
    assert on_disk == rows


def test_stops_after_the_unstable_row():
    sim = _Sim(unstable_at=200)
    rows = lbm.trace_run(sim, 1000, 100)
    assert [r["step"] for r in rows] == [0, 100, 200] and rows[-1]["status"] == 1
    assert sim.step == 200


def test_arguments_are_checked():
    with pytest.raises(ValueError):
        lbm.trace_run(_Sim(), 100, 0)
    assert [r["step"] for r in lbm.trace_run(_Sim(), 0, 10)] == [0]
