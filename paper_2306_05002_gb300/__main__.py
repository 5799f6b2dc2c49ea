"""Command line: advance one of the built-in synthetic workloads and report its diagnostics.

    python -m paper_2306_05002_gb300 drop --n 64 --p 3 --steps 500 --precision fp32bulk
    python -m paper_2306_05002_gb300 rt --n 256 --p 4 --steps 3
    python -m paper_2306_05002_gb300 slab --n 100 --p 3 --steps 1000 --precision fp64
    python -m paper_2306_05002_gb300 rk --n 64 --p 3 --steps 100 --elem tri
    python -m paper_2306_05002_gb300 rk --n 64 --p 3 --steps 2 --reinit 50
    python -m paper_2306_05002_gb300 rtpaper --steps 100 --save rt.npz
    python -m paper_2306_05002_gb300 --resume rt.npz --steps 100 --save rt.npz

Workloads (``workloads.py``): ``slab`` (1D periodic water slab in air), ``drop`` (2D periodic
water drop in air, seeded centre), ``rt`` (2D viscous Rayleigh-Taylor with walls, gravity and
surface tension), ``rtpaper`` (the paper's Rayleigh-Taylor domain with slip sides and the pressure
top), ``bubble`` (the paper's rising bubble, ``--case 1`` or ``2``), ``rk`` (the kinematic Rider-Kothe vortex, phi and psi only, classical RK4, on rectangles or,
with ``--elem tri``, triangles; prints phi's min/max and mean instead of ``dg_diag``).  The state is
built on the host (or read from a checkpoint with ``--resume``), moved to the GPU once, stepped
with ``dg_step`` in one call and read back; the line printed holds the wall time of the call and
the FP64 diagnostics of ``dg_diag`` (integrals of the seven variables, min/max of phi and P).
``--save`` writes the final state, the problem and the clock as a checkpoint
(``checkpoint.py``); ``--grad-lift`` selects BR1-lifted gradients (FP64 only).
"""
import argparse
import json
import time


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2306_05002_gb300")
    ap.add_argument("workload", nargs="?", default="drop", choices=["slab", "drop", "rt", "rtpaper", "bubble", "rk"])
    ap.add_argument("--case", type=int, default=1, choices=[1, 2], help="rising-bubble case (bubble only)")
    ap.add_argument("--n", type=int, default=None, help="elements per direction")
    ap.add_argument("--p", type=int, default=None, help="polynomial order")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--precision", choices=["fp64", "fp32bulk"], default="fp32bulk")
    ap.add_argument("--seed", type=int, default=None)
    ap.add_argument("--elem", choices=["quad", "tri"], default="quad", help="element type (rk only)")
    ap.add_argument("--reinit", type=int, default=0,
                    help="rk on rectangles: level-set re-initialisation steps after the time steps")
    ap.add_argument("--grad-lift", action="store_true", help="BR1-lifted gradients of phi and psi (fp64)")
    ap.add_argument("--resume", default=None, help="start from this checkpoint (the workload is ignored)")
    ap.add_argument("--save", default=None, help="write a checkpoint of the final state here")
    args = ap.parse_args(argv)

    import torch
    import paper_2306_05002_gb300 as dg
    from paper_2306_05002_gb300 import checkpoint as C
    from paper_2306_05002_gb300 import workloads as W

    t0_sim, step0 = 0.0, 0
    if args.resume:
        wl, state, t0_sim, step0, dt = C.load(args.resume)
        wl.dt = dt
        if isinstance(wl, W.KinWorkload):
            return _kinematic(args, {}, (wl, t0_sim, step0))
    else:
        kw = {}
        if args.p is not None:
            kw["p"] = args.p
        if args.workload == "rk":
            return _kinematic(args, kw)
        if args.workload == "slab":
            if args.n is not None:
                kw["nx"] = args.n
            wl = W.slab_1d(**kw)
        elif args.workload == "rtpaper":
            if args.n is not None:
                kw["nx"], kw["ny"] = args.n, 4 * args.n
            wl = W.rayleigh_taylor_paper(**kw)
        elif args.workload == "bubble":
            if args.n is not None:
                kw["nx"], kw["ny"] = args.n, 2 * args.n
            wl = W.rising_bubble(case=args.case, **kw)
        else:
            if args.n is not None:
                kw["n"] = args.n
            if args.seed is not None:
                kw["seed"] = args.seed
            wl = (W.drop_2d if args.workload == "drop" else W.rayleigh_taylor)(**kw)
        state = wl.w
    if args.grad_lift:
        wl.grad_lift = True

    s = dg.Solver(wl, precision=args.precision)
    w = torch.from_numpy(state.copy()).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.dg_step(w, wl.dt, args.steps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    status = s.dg_status_read()
    diag = s.dg_diag(w)
    s.close()
    if args.save:
        C.save(args.save, wl, w, t=t0_sim + args.steps * wl.dt, step=step0 + args.steps)
    print(json.dumps({"workload": wl.name, "nodes": wl.N, "steps": args.steps, "dt": wl.dt,
                      "precision": args.precision, "wall_s": wall, "device_status": status,
                      "t": t0_sim + args.steps * wl.dt, "step": step0 + args.steps,
                      "integrals": diag[:7], "phi_min_max": diag[7:9], "P_min_max": diag[9:11]}))
    return 0 if status == 0 else 1


def _kinematic(args, kw, resumed=None):
    import torch
    import paper_2306_05002_gb300 as dg
    from paper_2306_05002_gb300 import checkpoint as C
    from paper_2306_05002_gb300 import workloads as W
    if resumed is not None:
        wl, t_sim, step0 = resumed
    else:
        if args.n is not None:
            kw["n"] = args.n
        wl = W.rider_kothe(elem=args.elem, **kw)
        t_sim, step0 = 0.0, 0
    s = dg.KinematicSolver(wl)
    w = torch.from_numpy(wl.w.copy()).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.dg_kin_step(w, t_sim, wl.dt, args.steps)
    if args.reinit > 0:
        s.dg_reinit(w, args.reinit)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    status = s.dg_status_read()
    phi = w[0]
    out = {"workload": wl.name, "nodes": wl.N, "steps": args.steps, "dt": wl.dt, "precision": "fp64",
           "wall_s": wall, "device_status": status, "t": t_sim + args.steps * wl.dt,
           "step": step0 + args.steps, "phi_min_max": [phi.min().item(), phi.max().item()],
           "phi_mean": phi.mean().item()}
    s.close()
    if args.save:
        C.save(args.save, wl, w, t=t_sim + args.steps * wl.dt, step=step0 + args.steps)
    print(json.dumps(out))
    return 0 if status == 0 else 1


if __name__ == "__main__":
    raise SystemExit(main())
