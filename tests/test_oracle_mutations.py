"""Mutation check of the oracle's pins: each entry below plants one plausible mistake in a copy
of the oracle's C source (a dropped term, a flipped sign, a transposed operator, a one-sided
average, a wrong boundary ghost, a wrong Runge-Kutta coefficient, ...), builds the copy, and runs
the pins of ``tests/test_oracle_*.py`` against it.  Every mistake must make at least one pin fail:
a pin set that let one through would not tie the oracle to the paper at that point.

The mutated copies are compiled with the oracle's own flags; the pins of each copy run in a
separate (spawned) process through ``oracle.using``, which routes the oracle's functions to it.
"""
import importlib
import itertools
import multiprocessing
import os
import tempfile
from concurrent.futures import ProcessPoolExecutor, ThreadPoolExecutor

import pytest

import oracle

SRC = {name: os.path.join(os.path.dirname(oracle.__file__), name) for name in ("dg_oracle.c", "dg_oracle_tri.c")}

# (file, original text, planted mistake, what it models).  Each original text occurs exactly once.
MUTATIONS = [
    # closure (Sec. 2)
    ("dg_oracle.c", "q->P = (rhoe - (phi1 * g->C[0] + phi2 * g->C[1]))",
     "q->P = (rhoe + (phi1 * g->C[0] + phi2 * g->C[1]))", "stiffened-gas constant added, not removed"),
    ("dg_oracle.c", "q->c = sqrt(gam * (q->P + pinf) / q->rho);", "q->c = sqrt(gam * q->P / q->rho);",
     "sound speed without the mixture Pinf"),
    ("dg_oracle.c", "double rhoe = q->rE - 0.5 * (q->ru * q->ru + q->rv * q->rv) / q->rho;",
     "double rhoe = q->rE - (q->ru * q->ru + q->rv * q->rv) / q->rho;", "kinetic energy without 1/2"),
    ("dg_oracle.c", "q->B = pr->gamma[0] * (q->P + pr->pinf[0]) / (pr->gamma[0] - 1.0) -",
     "q->B = pr->gamma[0] * (q->P + pr->pinf[1]) / (pr->gamma[0] - 1.0) -", "B with the wrong phase's Pinf"),
    # operators
    ("dg_oracle.c", "wt[k] = 2.0 / (p * (p + 1.0) * P * P);", "wt[k] = 2.0 / (p * (p + 1.0) * P);",
     "GLL weight with P instead of P^2"),
    ("dg_oracle.c", "gr[0] = (aj == bj) ? (2.0 / g->hx) * g->D[ai * g->P1 + bi] : 0.0;",
     "gr[0] = (aj == bj) ? (2.0 / g->hx) * g->D[bi * g->P1 + ai] : 0.0;", "transposed derivative matrix"),
    ("dg_oracle.c", "gr[1] = (g->dim == 2 && ai == bi) ? (2.0 / g->hy) * g->D[aj * g->P1 + bj] : 0.0;",
     "gr[1] = (g->dim == 2 && ai == bi) ? (2.0 / g->hx) * g->D[aj * g->P1 + bj] : 0.0;",
     "y-derivative scaled by the x element width"),
    # normal, a_1, stress
    ("dg_oracle.c", "for (int d = 0; d < 2; ++d) t->n[d] = norm < 1e-12 ? 0.0 : t->gpsi[d] / norm;",
     "for (int d = 0; d < 2; ++d) t->n[d] = t->gpsi[d] / norm;", "no degenerate-normal branch"),
    ("dg_oracle.c", "t->a1[d] = Gam * (eps * t->gphi[d] - s * t->n[d]);",
     "t->a1[d] = Gam * (eps * t->gphi[d] + s * t->n[d]);", "sharpening term with the wrong sign"),
    ("dg_oracle.c", "t->tau[0][1] = t->tau[1][0] = mu * (t->gu[1] + t->gv[0]);",
     "t->tau[0][1] = t->tau[1][0] = mu * t->gu[1];", "shear stress without dv/dx"),
    ("dg_oracle.c", "t->tau[0][0] = 2.0 * mu * (t->gu[0] - div / 3.0);",
     "t->tau[0][0] = 2.0 * mu * (t->gu[0] - div / 2.0);", "wrong bulk part of the stress"),
    # volume fluxes and sources
    ("dg_oracle.c", "F[ORC_M2][d] = q->m2 * vel[d] + pr->rho0[1] * t->a1[d];",
     "F[ORC_M2][d] = q->m2 * vel[d] - pr->rho0[1] * t->a1[d];", "R_2 = +rho_2 a_1 (a_2 = -a_1 dropped)"),
    ("dg_oracle.c", "F[ORC_RU][d] = q->ru * vel[d] + (d == 0 ? q->P : 0.0) - drho0 * t->a1[d] * q->u;",
     "F[ORC_RU][d] = q->ru * vel[d] + (d == 0 ? q->P : 0.0) + drho0 * t->a1[d] * q->u;", "f (x) u with the wrong sign"),
    ("dg_oracle.c", "- drho0 * t->a1[d] * q->k - q->B * t->a1[d];", "- drho0 * t->a1[d] * q->k;",
     "energy flux without the enthalpy term B a_1"),
    ("dg_oracle.c", "F[ORC_RE][d] = (q->rE + q->P) * vel[d]", "F[ORC_RE][d] = q->rE * vel[d]",
     "energy flux without the pressure work"),
    ("dg_oracle.c", "add(&vol, ORC_PHI, n, -wa * tphi,", "add(&vol, ORC_PHI, n, wa * tphi,",
     "non-conservative transport of phi with the wrong sign"),
    ("dg_oracle.c", "double gu = q->rho * (pr->g[0] * q->u + pr->g[1] * q->v);",
     "double gu = q->rho * pr->g[0] * q->u;", "gravity work without its y part"),
    ("dg_oracle.c", "double s = pr->sigma * t->kappa * dG;", "double s = -pr->sigma * t->kappa * dG;",
     "surface-tension force with the wrong sign"),
    # face fluxes
    ("dg_oracle.c", "double lam = fmax(fabs(unm) + qm->c, fabs(unp) + qp->c);", "double lam = fabs(unm) + qm->c;",
     "one-sided Lax-Friedrichs speed"),
    ("dg_oracle.c", "double Fh = 0.5 * (Fcp[v] + Fcm[v]) - lam * hj;", "double Fh = 0.5 * (Fcp[v] + Fcm[v]) + lam * hj;",
     "anti-dissipative Lax-Friedrichs term"),
    ("dg_oracle.c", "add(&srf, v, nm, wf * (lam - unm) * hj,", "add(&srf, v, nm, wf * (lam + unm) * hj,",
     "transport flux with the wrong upwind sign"),
    ("dg_oracle.c", "double ahat = Gam * (eps * (gn + eta * jump) - sharp);\n          double amag",
     "double ahat = Gam * (eps * (gn - eta * jump) - sharp);\n          double amag", "SIP penalty with the wrong sign"),
    ("dg_oracle.c", "add(&srf, v, nb, -wf * Cq[v] * sym * gm,", "add(&srf, v, nb, wf * Cq[v] * sym * gm,",
     "SIP symmetric term with the wrong sign"),
    ("dg_oracle.c", "Cq[ORC_RE] = 0.5 * (qp->B + qm->B) + drho0 * 0.5 * (qp->k + qm->k);",
     "Cq[ORC_RE] = qm->B + drho0 * 0.5 * (qp->k + qm->k);", "one-sided B in the energy's face coefficient"),
    ("dg_oracle.c", "Cq[ORC_M2] = -pr->rho0[1];", "Cq[ORC_M2] = pr->rho0[1];", "face coefficient of m_2 with the wrong sign"),
    ("dg_oracle.c", "double Jf = g.dim == 2 ? 0.5 * (f < 2 ? g.hy : g.hx) : 1.0;\n      for (int k = 0; k < nk; ++k) {\n        int a = face_node(&g, f, k);\n        long nm = (long)e * Np + a;",
     "double Jf = g.dim == 2 ? 0.5 * (f < 2 ? g.hx : g.hy) : 1.0;\n      for (int k = 0; k < nk; ++k) {\n        int a = face_node(&g, f, k);\n        long nm = (long)e * Np + a;",
     "face Jacobians of x- and y-faces swapped"),
    ("dg_oracle.c", "double th_x = 0.5 * (tp_m[0] + tm_m[0]) + eta * mu_avg * (qp->u - qm->u);",
     "double th_x = 0.5 * (tp_m[0] + tm_m[0]) + eta * mu_avg * (qm->u - qp->u);", "viscous penalty with the wrong sign"),
    ("dg_oracle.c", "double eh = 0.5 * (tu_p + tu_m) + eta * mu_avg * (qp->k - qm->k);",
     "double eh = tu_m + eta * mu_avg * (qp->k - qm->k);", "one-sided viscous work at faces"),
    # boundaries (Sec. 4.2)
    ("dg_oracle.c", "int slip = pr->bc[f] == ORC_BC_SLIP;", "int slip = 0;", "slip walls reverse the whole velocity"),
    ("dg_oracle.c", "ghost.q.ru = tm->q.ru - 2.0 * un * m[0];\n            ghost.q.rv = tm->q.rv - 2.0 * un * m[1];",
     "ghost.q.ru = tm->q.ru;\n            ghost.q.rv = tm->q.rv;", "slip walls reverse no momentum"),
    ("dg_oracle.c", "double un = tm->q.ru * m[0] + tm->q.rv * m[1];", "double un = tm->q.ru * m[1] + tm->q.rv * m[0];",
     "slip walls reverse the tangential momentum"),
    ("dg_oracle.c", "          ghost = *tm;\n",
     "          ghost = *tm;\n          for (int d = 0; d < 2; ++d) { ghost.tau[d][0] = -tm->tau[d][0]; ghost.tau[d][1] = -tm->tau[d][1]; }\n",
     "wall ghost stress reversed instead of equal to the own"),
    ("dg_oracle.c", "pr->p_bc[f] * (ph1 * g.gi[0] + ph2 * g.gi[1]) + (ph1 * g.C[0] + ph2 * g.C[1])};",
     "pr->p_bc[f] * (ph1 * g.gi[0] + ph2 * g.gi[1])};", "pressure-boundary energy without the stiffened-gas constant"),
    # mass matrix, time stepping, diagnostics
    ("dg_oracle.c", "      double Minv = 1.0 / (node_weight(&g, a) * g.J);\n      for (int v = 0; v < NV; ++v) {",
     "      double Minv = 1.0 / node_weight(&g, a);\n      for (int v = 0; v < NV; ++v) {", "M^-1 without the Jacobian"),
    ("dg_oracle.c", "w2[i] = 0.75 * w[i] + 0.25 * (w1[i] + dt * L[i]);", "w2[i] = 0.5 * w[i] + 0.5 * (w1[i] + dt * L[i]);",
     "wrong second SSP-RK3 stage"),
    ("dg_oracle.c", "w[i] = w[i] / 3.0 + 2.0 / 3.0 * (w2[i] + dt * L[i]);",
     "w[i] = w[i] / 3.0 + 2.0 / 3.0 * (w2[i] + 0.5 * dt * L[i]);", "wrong third SSP-RK3 stage"),
    ("dg_oracle.c", "out[v] += wJ * wn[v];", "out[v] += wn[v];", "diagnostic integrals without quadrature weights"),
    # BR1-lifted gradients (option grad_lift)
    ("dg_oracle.c", "double lift = wf / (node_weight(g, a) * g->J) * 0.5 * (f[np_] - f[nm]);",
     "double lift = wf / (node_weight(g, a) * g->J) * (f[np_] - f[nm]);", "lifting with the full jump"),
    ("dg_oracle.c", "gx[nm] += lift * m[0];", "gx[nm] -= lift * m[0];", "lifting against the outward normal"),
    ("dg_oracle.c", "double tphi = q->u * t->bphi[0] + q->v * t->bphi[1];",
     "double tphi = q->u * t->gphi[0] + q->v * t->gphi[1];", "transport of phi on the lifted gradient"),
    # kinematic mode (Sec. 4.1)
    ("dg_oracle.c", "k->a1[d] = Gam * (eps * k->gphi[d] - s * k->n[d]);", "k->a1[d] = Gam * (eps * k->gphi[d] + s * k->n[d]);",
     "kinematic sharpening term with the wrong sign"),
    ("dg_oracle.c", "add(&ac, 0, nm, wf * (lam - unm) * hj_phi,", "add(&ac, 0, nm, wf * (lam + unm) * hj_phi,",
     "kinematic transport flux with the wrong upwind sign"),
    ("dg_oracle.c", "for (size_t i = 0; i < len; ++i) { acc[i] += 2.0 * k[i]; ws[i] = w[i] + dt * k[i]; }\n    if (rc == 0) rc = orc_kin_rhs",
     "for (size_t i = 0; i < len; ++i) { acc[i] += k[i]; ws[i] = w[i] + dt * k[i]; }\n    if (rc == 0) rc = orc_kin_rhs",
     "RK4 weight of the third stage"),
    ("dg_oracle.c", "va -= psi[(long)e * Np + b] * gr[0];", "va += psi[(long)e * Np + b] * gr[0];",
     "vortex velocity from the stream function with the wrong sign of v"),
    ("dg_oracle.c", "ua += psi[(long)e * Np + b] * gr[1];", "ua += psi[(long)e * Np + b] * gr[0];",
     "vortex velocity from the wrong derivative of the stream function"),
    ("dg_oracle.c", "return sx * sx * sy * sy * cos(M_PI * t / vel->T) / M_PI;",
     "return sx * sx * sy * sy * cos(M_PI * t / vel->T);", "stream function without its 1/pi"),
    # re-initialisation (end of Sec. 3)
    ("dg_oracle.c", "R[nk] += wk * S[nk] * (1.0 - gm);", "R[nk] += wk * S[nk] * (gm - 1.0);",
     "re-initialisation source with the printed (growing) sign"),
    ("dg_oracle.c", "else S[n] = tanh(p0[n] / (2.0 * pr->eps * gm));", "else S[n] = tanh(p0[n] / (pr->eps * gm));",
     "smeared sign without the factor 2"),
    ("dg_oracle.c", "if (gmb != 0.0) R[(long)e * Np + b] += -wf * 0.5 * nu * jump * gmb;",
     "if (gmb != 0.0) R[(long)e * Np + b] += wf * 0.5 * nu * jump * gmb;", "re-initialisation symmetric term sign"),
    # triangles (mesh (b))
    ("dg_oracle_tri.c", "double eta = pr->c_ip * (pr->p + 1.0) * (pr->p + 2.0) / he;",
     "double eta = -pr->c_ip * (pr->p + 1.0) * (pr->p + 2.0) / he;", "triangle SIP penalty with the wrong sign"),
    ("dg_oracle_tri.c", "double fphi = (lam - unm) * 0.5 * jump + ahat;", "double fphi = (lam - unm) * jump + ahat;",
     "triangle transport flux with the full jump"),
    ("dg_oracle_tri.c", "Rp[n] += wf * (l[n] * fphi - sym * glm);", "Rp[n] += wf * (l[n] * fphi + sym * glm);",
     "triangle symmetric term with the wrong sign"),
    ("dg_oracle_tri.c", "o->a1[d] = pr->Gamma * (pr->eps * o->gphi[d] - sp * o->n[d]);",
     "o->a1[d] = pr->Gamma * (pr->eps * o->gphi[d] + sp * o->n[d]);", "triangle sharpening term with the wrong sign"),
    ("dg_oracle_tri.c", "double wf = T.gw[k] * 0.5 * len;", "double wf = T.gw[k] * len;", "triangle edge Jacobian doubled"),
    ("dg_oracle_tri.c", "for (size_t i = 0; i < len; ++i) w[i] = w[i] + dt / 6.0 * (acc[i] + k[i]);",
     "for (size_t i = 0; i < len; ++i) w[i] = w[i] + dt / 6.0 * (acc[i] + 2.0 * k[i]);", "triangle RK4 last weight"),
    ("dg_oracle_tri.c", "Rs[n] += -wq * l[n] * ts;", "Rs[n] += wq * l[n] * ts;", "triangle level-set transport sign"),
]

# The pin modules, cheapest first (a mutant is usually caught by an early one).
PIN_MODULES = ["test_oracle_operators", "test_oracle_closure", "test_oracle_walls", "test_oracle_lifting",
               "test_oracle_invariants",
               "test_oracle_pressure_bc", "test_oracle_reinit", "test_oracle_kinematic", "test_oracle_triangles",
               "test_oracle_convergence"]


def _pins():
    """Every pin of the oracle test modules as (name, callable, kwargs), parametrisations expanded."""
    out = []
    for modname in PIN_MODULES:
        mod = importlib.import_module(f"tests.{modname}")
        for name in sorted(n for n in dir(mod) if n.startswith("test_")):
            fn = getattr(mod, name)
            grids = []
            for mark in getattr(fn, "pytestmark", []):
                if mark.name != "parametrize":
                    continue
                names, values = mark.args[0], mark.args[1]
                names = [s.strip() for s in names.split(",")] if isinstance(names, str) else list(names)
                grids.append([dict(zip(names, v if len(names) > 1 else (v,))) for v in values])
            for combo in itertools.product(*grids) if grids else [()]:
                kw = {}
                for d in combo:
                    kw.update(d)
                out.append((f"{modname}.{name}{kw or ''}", fn, kw))
    return out


def _mutated_source(fname, old, new):
    text = open(SRC[fname]).read()
    assert text.count(old) == 1, f"{fname}: the original text of a mutation must occur exactly once: {old!r}"
    return text.replace(old, new)


def test_mutation_originals_occur_once():
    for fname, old, new, what in MUTATIONS:
        _mutated_source(fname, old, new)


def _first_failing_pin(path):
    """Run the pins against the oracle build at `path`; the name of the first that fails, or None."""
    with oracle.using(path):
        for name, fn, kw in _pins():
            try:
                fn(orc=oracle, **kw)
            except Exception:  # an assertion, or an error the mistake provoked
                return name
    return None


@pytest.mark.slow
def test_every_planted_mistake_is_caught_by_a_pin():
    assert len(_pins()) > 60
    workers = min(8, os.cpu_count() or 2)
    with tempfile.TemporaryDirectory() as tmp:
        def build(k):
            fname, old, new, _ = MUTATIONS[k]
            d = os.path.join(tmp, f"m{k}")
            os.makedirs(d)
            srcs = []
            for name, path in SRC.items():
                dst = os.path.join(d, name)
                with open(dst, "w") as fh:
                    fh.write(_mutated_source(fname, old, new) if name == fname else open(path).read())
                srcs.append(dst)
            out = os.path.join(d, "liboracle_mut.so")
            oracle.compile_sources(srcs, out, include_dir=os.path.dirname(oracle.__file__))
            return out

        with ThreadPoolExecutor(max_workers=workers) as ex:
            libs = list(ex.map(build, range(len(MUTATIONS))))
        # the pins of different mutants run in separate processes (spawned: no GPU state is shared)
        with ProcessPoolExecutor(max_workers=workers, mp_context=multiprocessing.get_context("spawn")) as ex:
            caught = list(ex.map(_first_failing_pin, libs))
    missed = [m[3] for m, c in zip(MUTATIONS, caught) if c is None]
    assert not missed, f"planted mistakes no pin catches: {missed}"
