"""Checkpoint and resume of a time integration: one problem's description, state and clock in one
``.npz`` file (or a batch of problems in one file).

A context of the library keeps no solution state between calls: the caller's array is the state,
and what a context holds besides (operator tables, captured step graphs, workspaces) is rebuilt from
the problem description when a context is created.  So a checkpoint is the state array plus what
re-creates the context (the fields of the problem's ``Workload`` or ``KinWorkload``), the time, the
step count and the step size.  Files are written to a temporary name and renamed, so an interrupted
save leaves the previous checkpoint intact.
"""
from __future__ import annotations

import dataclasses
import json
import os

import numpy as np

from . import workloads as W

FORMAT = 1
_KINDS = {"Workload": W.Workload, "KinWorkload": W.KinWorkload}


def _host(state) -> np.ndarray:
    """A float64 host copy of a numpy array or a torch tensor on any device."""
    if hasattr(state, "detach"):
        state = state.detach().to("cpu").numpy()
    a = np.array(state, dtype=np.float64, copy=True)
    if a.ndim != 2:
        raise ValueError("a state is a (fields, nodes) array")
    return a


def _describe(problem) -> str:
    kind = type(problem).__name__
    if kind not in _KINDS:
        raise TypeError(f"cannot checkpoint a {kind}: expected Workload or KinWorkload")
    fields = {f.name: getattr(problem, f.name) for f in dataclasses.fields(problem) if f.name != "w"}
    return json.dumps({"kind": kind, "fields": fields}, default=_jsonable)


def _jsonable(x):
    if isinstance(x, np.generic):
        return x.item()
    if isinstance(x, np.ndarray):
        return x.tolist()
    raise TypeError(f"field value {x!r} is not serialisable")


def _rebuild(desc: str, state: np.ndarray):
    d = json.loads(desc)
    cls = _KINDS[d["kind"]]
    names = {f.name for f in dataclasses.fields(cls)}
    fields = {k: (tuple(v) if isinstance(v, list) else v) for k, v in d["fields"].items() if k in names}
    problem = cls(**fields)
    problem.w = state
    nf, n = (2 if cls is W.KinWorkload else 7), problem.N
    if state.shape != (nf, n):
        raise ValueError(f"state of shape {state.shape} does not fit the problem ({nf}, {n})")
    return problem


def _write(path: str, **arrays) -> None:
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "wb") as f:
        np.savez(f, **arrays)
    os.replace(tmp, path)


def save(path: str, problem, state, *, t: float = 0.0, step: int = 0, dt: float | None = None) -> None:
    """Write one problem, its state (numpy array or torch tensor, any device) and its clock."""
    s = _host(state)
    _rebuild(_describe(problem), s)  # refuse a state that does not fit the problem
    _write(path, format=np.int64(FORMAT), problem=np.array(_describe(problem)), state=s,
           t=np.float64(t), step=np.int64(step), dt=np.float64(problem.dt if dt is None else dt))


def load(path: str):
    """(problem, state, t, step, dt) from a file written by `save`; the problem's ``w`` is the state."""
    with np.load(path, allow_pickle=False) as z:
        if int(z["format"]) != FORMAT or "state" not in z:
            raise ValueError(f"{path}: not a single-problem checkpoint of format {FORMAT}")
        state = np.array(z["state"], dtype=np.float64)
        problem = _rebuild(str(z["problem"]), state)
        return problem, state, float(z["t"]), int(z["step"]), float(z["dt"])


def save_batch(path: str, problems, states, *, t: float = 0.0, step: int = 0) -> None:
    """Write a batch of problems (each with its own step size) and their states."""
    if len(problems) != len(states) or not problems:
        raise ValueError("need one state per problem")
    arrays = {"format": np.int64(FORMAT), "count": np.int64(len(problems)), "t": np.float64(t),
              "step": np.int64(step), "dts": np.array([wl.dt for wl in problems], dtype=np.float64)}
    for k, (wl, st) in enumerate(zip(problems, states)):
        s = _host(st)
        _rebuild(_describe(wl), s)
        arrays[f"problem{k}"] = np.array(_describe(wl))
        arrays[f"state{k}"] = s
    _write(path, **arrays)


def load_batch(path: str):
    """(problems, states, t, step) from a file written by `save_batch`."""
    with np.load(path, allow_pickle=False) as z:
        if int(z["format"]) != FORMAT or "count" not in z:
            raise ValueError(f"{path}: not a batch checkpoint of format {FORMAT}")
        problems, states = [], []
        for k in range(int(z["count"])):
            s = np.array(z[f"state{k}"], dtype=np.float64)
            wl = _rebuild(str(z[f"problem{k}"]), s)
            wl.dt = float(z["dts"][k])
            problems.append(wl)
            states.append(s)
        return problems, states, float(z["t"]), int(z["step"])
