"""Checkpoint files (paper_2306_05002_gb300.checkpoint): a save/load round trip restores the problem
description, the state bit for bit and the clock, for single problems of both kinds and for a batch;
a state that does not fit its problem, and a file of another kind, are refused.  On the GPU, a run
resumed from a checkpoint continues exactly as the uninterrupted run."""
import os

import numpy as np
import pytest

from paper_2306_05002_gb300 import checkpoint as C
from paper_2306_05002_gb300 import workloads as W


def test_round_trip_full_model(tmp_path):
    wl = W.rayleigh_taylor_paper(nx=2, ny=6, p=3)
    state = wl.w + 1e-3 * np.random.default_rng(1).standard_normal(wl.w.shape)
    path = os.path.join(tmp_path, "rt.npz")
    C.save(path, wl, state, t=0.125, step=17)
    got, s, t, step, dt = C.load(path)
    assert np.array_equal(s.view(np.uint64), state.view(np.uint64))
    assert (t, step, dt) == (0.125, 17, wl.dt)
    assert got.problem_kwargs() == wl.problem_kwargs()
    assert got.name == wl.name and got.nsteps == wl.nsteps and got.w is s


def test_round_trip_kinematic_triangles(tmp_path):
    wl = W.rider_kothe(n=4, p=2, elem="tri")
    path = os.path.join(tmp_path, "kin.npz")
    C.save(path, wl, wl.w, t=1.5, step=3, dt=2e-3)
    got, s, t, step, dt = C.load(path)
    assert np.array_equal(s, wl.w) and (t, step, dt) == (1.5, 3, 2e-3)
    assert got.elem == "tri" and got.velocity_kwargs() == wl.velocity_kwargs()
    assert got.problem_kwargs() == wl.problem_kwargs()


def test_round_trip_batch(tmp_path):
    wls = W.ensemble(n=3, seed=4, nmin=4, nmax=6)
    path = os.path.join(tmp_path, "batch.npz")
    C.save_batch(path, wls, [wl.w for wl in wls], t=0.5, step=9)
    got, states, t, step = C.load_batch(path)
    assert (t, step) == (0.5, 9) and len(got) == 3
    for a, b, s in zip(wls, got, states):
        assert a.problem_kwargs() == b.problem_kwargs() and a.dt == b.dt and a.name == b.name
        assert np.array_equal(s, a.w)


def test_refusals(tmp_path):
    wl = W.drop_2d(n=3, p=2, seed=1)
    with pytest.raises(ValueError):
        C.save(os.path.join(tmp_path, "bad.npz"), wl, wl.w[:, :-1])
    path = os.path.join(tmp_path, "batch.npz")
    C.save_batch(path, [wl], [wl.w])
    with pytest.raises(ValueError):
        C.load(path)
    with pytest.raises(TypeError):
        C.save(os.path.join(tmp_path, "x.npz"), {"nx": 3}, wl.w)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32bulk"])
def test_resume_continues_the_run(dg, tmp_path, precision):
    """10 steps in one run against 4 steps, a checkpoint, a new context from the file and 6 more
    steps: bit for bit in FP64 (the same kernels on the same state); FP32-bulk, whose call boundary
    takes the carried float pair back to FP64, within 1e-12 of the state's scale."""
    import torch
    wl = W.drop_2d(n=8, p=3, seed=2)
    s = dg.Solver(wl, precision=precision)
    a = torch.from_numpy(wl.w.copy()).cuda()
    s.dg_step(a, wl.dt, 10)
    b = torch.from_numpy(wl.w.copy()).cuda()
    s.dg_step(b, wl.dt, 4)
    s.close()
    path = os.path.join(tmp_path, "run.npz")
    C.save(path, wl, b, t=4 * wl.dt, step=4)
    wl2, st, t, step, dt = C.load(path)
    s2 = dg.Solver(wl2, precision=precision)
    c = torch.from_numpy(st).cuda()
    s2.dg_step(c, dt, 10 - step)
    s2.close()
    x, y = a.cpu().numpy(), c.cpu().numpy()
    if precision == "fp64":
        assert np.array_equal(x, y)
    else:
        for v in range(7):
            assert np.abs(x[v] - y[v]).max() <= 1e-12 * np.abs(x[v]).max() + 1e-300, v


@pytest.mark.gpu
def test_command_line_save_and_resume(dg, tmp_path):
    """`python -m paper_2306_05002_gb300 ... --save` then `--resume ... --save`: 4 + 6 steps give the
    state of 10 steps in one run, bit for bit (FP64), and the clock adds up."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    run = lambda *a: subprocess.run([sys.executable, "-m", "paper_2306_05002_gb300", *a], cwd=root,
                                    capture_output=True, text=True, timeout=300)
    a, b = os.path.join(tmp_path, "a.npz"), os.path.join(tmp_path, "b.npz")
    base = ["drop", "--n", "8", "--p", "3", "--precision", "fp64"]
    r1 = run(*base, "--steps", "4", "--save", a)
    r2 = run("--resume", a, "--steps", "6", "--precision", "fp64", "--save", a)
    r3 = run(*base, "--steps", "10", "--save", b)
    for r in (r1, r2, r3):
        assert r.returncode == 0, r.stderr[-2000:]
    assert json.loads(r2.stdout.splitlines()[-1])["step"] == 10
    _, sa, ta, na, _ = C.load(a)
    _, sb, tb, nb, _ = C.load(b)
    assert np.array_equal(sa, sb) and na == nb == 10 and abs(ta - tb) <= 1e-15 * tb
