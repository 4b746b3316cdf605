"""The JSONL run log (paper_2511_00445_gb300/runlog.py): line layout and step
bookkeeping with a stand-in context on the CPU, and a short logged run on the
GPU whose lines carry the library's own observables."""
import json

import numpy as np
import pytest

from paper_2511_00445_gb300 import _binding as B
from paper_2511_00445_gb300 import runlog


class FakeContext:
    """Host stand-in with the observable calls the log makes."""

    def __init__(self, params):
        self.params = list(params)
        self.batch = len(self.params)
        self.steps = 0

    def step(self, n):
        self.steps += n

    def sync(self):
        pass

    def step_count(self):
        return self.steps

    def conserved(self, inst, check=True):
        return np.array([100.0 + inst, 1.0, 2.0, 0.5, -0.5, 0.0, 0.0, 0.0])

    def phase_difference(self, inst):
        return np.arange(6, dtype=float) + inst

    def energy_spectrum(self, inst):
        return np.zeros(4), 0.25 * (1 + self.steps)

    def phi_stats(self, inst):
        return 0.5, 0.01

    def length_scale(self, inst):
        return 3.0 + self.steps


def test_lines_and_steps(tmp_path):
    ps = [B.SolverParams(nx=8, ny=8, zeta=0.0), B.SolverParams(nx=8, ny=8, zeta=0.01)]
    tf = FakeContext(ps)
    path = tmp_path / "run.jsonl"
    n = runlog.run_logged(tf, steps=25, every=10, path=str(path))
    lines = [json.loads(s) for s in path.read_text().splitlines()]
    assert n == len(lines) == 2 * 4                       # steps 0, 10, 20, 25
    assert [ln["step"] for ln in lines[::2]] == [0, 10, 20, 25]
    assert [ln["instance"] for ln in lines[:2]] == [0, 1]
    first, last = lines[0], lines[-1]
    assert "mlups" not in first and last["mlups"] > 0
    assert last["hbm_gbs"] == pytest.approx(last["mlups"] * 168e-3)
    assert last["params"]["zeta"] == 0.01 and last["params"]["nx"] == 8
    assert last["sum_phi"] == 101.0 and last["momentum"] == [0.5, -0.5]
    assert last["L"] == 28.0 and last["E"] == pytest.approx(0.25 * 26)
    assert last["delta_u_rms"] == 1.0 and last["wc_rms"] == 6.0
    runlog.run_logged(tf, steps=0, every=5, path=str(path), append=True)
    assert len(path.read_text().splitlines()) == 10       # appended the step-25 lines again
    with pytest.raises(ValueError):
        runlog.run_logged(tf, steps=5, every=0, path=str(path))


@pytest.mark.gpu
def test_logged_gpu_run(tmp_path):
    ps = [B.SolverParams(nx=64, ny=64, zeta=0.005), B.SolverParams(nx=64, ny=64, zeta=0.01)]
    tf = B.TwoFluid(ps)
    tf.init_fields(3, phi0=0.5, dphi=0.01, S0=0.01)
    path = tmp_path / "gpu.jsonl"
    assert runlog.run_logged(tf, steps=20, every=10, path=str(path)) == 6
    lines = [json.loads(s) for s in path.read_text().splitlines()]
    for inst in (0, 1):
        mine = [ln for ln in lines if ln["instance"] == inst]
        assert [ln["step"] for ln in mine] == [0, 10, 20]
        s0 = mine[0]["sum_phi"]
        assert all(abs(ln["sum_phi"] - s0) <= 1e-9 * abs(s0) for ln in mine)   # phi mass conserved
        assert all(ln["nonfinite"] == 0 and ln["L"] > 0 and ln["E"] >= 0 for ln in mine)
        assert all(ln["mlups"] > 0 for ln in mine[1:])
        # the logged values are the library's own observables of the final state
        # (the shell histogram behind L sums within a block by FP64 shared-memory
        # atomics, so two evaluations agree to rounding, not bit for bit)
        assert mine[-1]["L"] == pytest.approx(tf.length_scale(inst), rel=1e-12)
        assert mine[-1]["sum_phi"] == tf.conserved(inst)[0]
    tf.close()
