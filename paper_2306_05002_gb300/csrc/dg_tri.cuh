// dg_tri.cuh -- kinematic mode (Sec. 4.1) on triangular elements, the paper's
// mesh (b): every cell of an nx x ny periodic Cartesian grid split along its
// rising diagonal into a lower-right triangle (type 0, vertices (x_i, y_j),
// (x_i+1, y_j), (x_i+1, y_j+1)) and an upper-left one (type 1, vertices
// (x_i, y_j), (x_i+1, y_j+1), (x_i, y_j+1)); element 2 (i + nx j) + type.
// FP64 (GB300, sm_103a).
//
// The same equations as dg_kin.cuh,
//   d(phi)/dt + u . grad(phi) = div a_1,   a_1 = Gamma (eps grad phi - phi (1 - phi) n),
//   d(psi)/dt + u . grad(psi) = 0,
// with a nodal basis of degree p on the equispaced nodes of each triangle. A
// triangle has no tensor-product structure and no collocated quadrature, so
// the weak form is integrated with a collapsed Gauss-Legendre rule of (p+2)^2
// points and (p+2)-point Gauss-Legendre edge rules, and L = M^-1 R with the
// full element mass matrix.  Fluxes as on quadrilaterals: transport
// (lambda - m.u-) [[f]] with lambda = max(|u-.m|, |u+.m|), and the SIP flux of
// a_1 with its symmetric term, penalty eta = c_ip (p+1)(p+2) / h_e with
// h_e = 2 |T| / |e|.
//
// One kernel per Runge-Kutta stage.  A persistent grid walks groups of EPB
// triangles; each CTA stages the reference tables (basis values and
// derivatives at the volume and edge points, the inverse reference mass matrix)
// in shared memory once, then per group: the own and neighbour nodal values,
// the integrand coefficients at every volume and edge point (one thread per
// point), the weak-form sums (one thread per node) and M^-1 with the stage
// update (one thread per node).  Neighbour values are read from the stage
// input, which no stage writes, so the stages need no other synchronisation
// than stream order.  FP64 is the bound, so what does not change between
// stages is computed once: the geometry of the two triangle types (host) and
// the spatial factor of the velocity at every quadrature point (device, at
// creation) -- the trigonometric functions would otherwise cost as much as the
// scheme itself.
#pragma once

#include <vector>

#include "dg_kin.cuh"

namespace dgpf {

// Reference-table layout of order p, in doubles (built by tri_tables).
struct TriLayout {
  int P1, NP, NQ1, NQV, NQE;
  __host__ __device__ constexpr explicit TriLayout(int p)
      : P1(p + 1), NP((p + 1) * (p + 2) / 2), NQ1(p + 2), NQV((p + 2) * (p + 2)), NQE(3 * (p + 2)) {}
  // basis values and reference derivatives at the volume points, [q][n]
  __host__ __device__ constexpr int bv() const { return 0; }
  __host__ __device__ constexpr int brv() const { return bv() + NQV * NP; }
  __host__ __device__ constexpr int bsv() const { return brv() + NQV * NP; }
  // at the edge points [f NQ1 + k], of the p+1 nodes of edge f only (tri_edge_node): the basis
  // values and their derivative d/dt along the edge (t in [-1, 1] from its first vertex to its
  // second); every other node's basis function vanishes on the edge, with its tangential
  // derivative
  __host__ __device__ constexpr int bev() const { return bsv() + NQV * NP; }
  __host__ __device__ constexpr int bet() const { return bev() + NQE * P1; }
  // physical derivative of every basis function along the outward normal of the edge, per
  // triangle type, [type][f NQ1 + k][n]
  __host__ __device__ constexpr int bn() const { return bet() + NQE * P1; }
  // inverse of the reference mass matrix sum_q w_q l_i l_j, [i][j]
  __host__ __device__ constexpr int minv() const { return bn() + 2 * NQE * NP; }
  // volume weights (collapsed factor included) and points
  __host__ __device__ constexpr int wv() const { return minv() + NP * NP; }
  __host__ __device__ constexpr int rv() const { return wv() + NQV; }
  __host__ __device__ constexpr int sv() const { return rv() + NQV; }
  // edge weights on [-1, 1] and edge points
  __host__ __device__ constexpr int we() const { return sv() + NQV; }
  __host__ __device__ constexpr int re() const { return we() + NQ1; }
  __host__ __device__ constexpr int se() const { return re() + NQE; }
  __host__ __device__ constexpr int size() const { return se() + NQE; }
};

// Index of the m-th node of edge f -- node (m, 0) of edge 0 (s = -1), (p - m, m) of edge 1
// (r + s = 0), (0, m) of edge 2 (r = -1) -- in the j-major node order, where node (i, j) sits at
// j (p+1) - j (j-1)/2 + i.
__host__ __device__ constexpr int tri_edge_node(int p, int f, int m) {
  return (f == 0 ? 0 : m) * (p + 1) - (f == 0 ? 0 : m) * ((f == 0 ? 0 : m) - 1) / 2 +
         (f == 0 ? m : (f == 1 ? p - m : 0));
}

template <int P>
struct TriGeom {
  static constexpr TriLayout L{P};
  static constexpr int NP = L.NP, NQ1 = L.NQ1, NQV = L.NQV, NQE = L.NQE;
  static constexpr int EPB = P >= 4 ? 6 : 8;
  static constexpr int THREADS = 128;
};


// Counter-clockwise vertices of triangle e (cell (i, j), type e & 1).
__device__ __forceinline__ void tri_vertices(const KinParams &kp, int e, double v[3][2]) {
  const int cell = e >> 1, type = e & 1;
  const double x0 = kp.x0 + (cell % kp.nx) * kp.hx, y0 = kp.y0 + (cell / kp.nx) * kp.hy;
  v[0][0] = x0;
  v[0][1] = y0;
  v[1][0] = x0 + kp.hx;
  v[1][1] = type == 0 ? y0 : y0 + kp.hy;
  v[2][0] = type == 0 ? x0 + kp.hx : x0;
  v[2][1] = y0 + kp.hy;
}

// Periodic neighbour across edge f (0: v1 v2, 1: v2 v3, 2: v3 v1) and its edge index.
// Type 0: bottom, right, diagonal; type 1: diagonal, top, left.
__device__ __forceinline__ int tri_neighbour(const KinParams &kp, int e, int f, int *f2) {
  const int cell = e >> 1, type = e & 1;
  const int ci = cell % kp.nx, cj = cell / kp.nx;
  if (type == 0) {
    if (f == 0) { *f2 = 1; return 2 * (ci + kp.nx * (cj > 0 ? cj - 1 : kp.ny - 1)) + 1; }
    if (f == 1) { *f2 = 2; return 2 * ((ci + 1 < kp.nx ? ci + 1 : 0) + kp.nx * cj) + 1; }
    *f2 = 0;
    return e + 1;
  }
  if (f == 0) { *f2 = 2; return e - 1; }
  if (f == 1) { *f2 = 0; return 2 * (ci + kp.nx * (cj + 1 < kp.ny ? cj + 1 : 0)); }
  *f2 = 1;
  return 2 * ((ci > 0 ? ci - 1 : kp.nx - 1) + kp.nx * cj);
}

// The velocity table of the triangles (kin_velocity_factor): U at every volume and edge point of
// every triangle, [e][NQV + NQE][2], volume points first.
template <int P>
__global__ void k_tri_velocity_table(const KinParams kp, double *__restrict__ tab) {
  using G = TriGeom<P>;
  constexpr TriLayout L = G::L;
  constexpr int NPT = G::NQV + G::NQE;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)kp.E * NPT) return;
  const int e = (int)(i / NPT), q = (int)(i % NPT);
  double v[3][2];
  tri_vertices(kp, e, v);
  const double r = q < G::NQV ? kp.ops[L.rv() + q] : kp.ops[L.re() + q - G::NQV];
  const double s = q < G::NQV ? kp.ops[L.sv() + q] : kp.ops[L.se() + q - G::NQV];
  const double x = v[0][0] + 0.5 * (1.0 + r) * (v[1][0] - v[0][0]) + 0.5 * (1.0 + s) * (v[2][0] - v[0][0]);
  const double y = v[0][1] + 0.5 * (1.0 + r) * (v[1][1] - v[0][1]) + 0.5 * (1.0 + s) * (v[2][1] - v[0][1]);
  kin_velocity_factor(kp, x, y, &tab[2 * i], &tab[2 * i + 1]);
}

template <int P>
cudaError_t launch_tri_velocity_table(const KinParams &kp, double *tab, cudaStream_t s) {
  constexpr int NPT = TriGeom<P>::NQV + TriGeom<P>::NQE;
  const long n = (long)kp.E * NPT;
  k_tri_velocity_table<P><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(kp, tab);
  return cudaGetLastError();
}

// phi, psi, their physical gradients and a_1 at one point, from the nodal values and the basis
// rows (values, r- and s-derivatives) of a triangle of constants g.
struct TriPoint {
  double phi, psi, gp[2], gs[2], n[2], a1[2];
};

template <int NP, bool PSI_VALUE>
__device__ __forceinline__ void tri_eval_point(const KinParams &kp, const TriConst &g, const double *fphi,
                                               const double *fpsi, const double *B, const double *Br,
                                               const double *Bs, TriPoint *o) {
  double ph = 0.0, ps = 0.0, pr = 0.0, pq = 0.0, sr = 0.0, sq = 0.0;
#pragma unroll
  for (int n = 0; n < NP; ++n) {
    ph = fma(B[n], fphi[n], ph);
    if (PSI_VALUE) ps = fma(B[n], fpsi[n], ps);  // psi itself is needed at the edges only
    pr = fma(Br[n], fphi[n], pr);
    pq = fma(Bs[n], fphi[n], pq);
    sr = fma(Br[n], fpsi[n], sr);
    sq = fma(Bs[n], fpsi[n], sq);
  }
  o->phi = ph;
  o->psi = ps;
  o->gp[0] = pr * g.rx + pq * g.sx;
  o->gp[1] = pr * g.ry + pq * g.sy;
  o->gs[0] = sr * g.rx + sq * g.sx;
  o->gs[1] = sr * g.ry + sq * g.sy;
  const double g2 = o->gs[0] * o->gs[0] + o->gs[1] * o->gs[1];
  const double rn = g2 < 1e-24 ? 0.0 : rsqrt(g2);  // n = 0 where |grad psi| < 1e-12
  const double sp = ph * (1.0 - ph);
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    o->n[d] = o->gs[d] * rn;
    o->a1[d] = kp.Gamma * (kp.eps * o->gp[d] - sp * o->n[d]);
  }
}

// phi, psi, d(phi)/dm and n . m at one edge point, m = sgn x the outward normal of the
// triangle's edge f (sgn = -1: a neighbour's trace, seen along the normal of the triangle being
// updated).  ihl: the reciprocal of half the edge length (d/dtau = hl d/dt along the edge; a
// product, not a division, on the FP64 pipe that bounds the kernel).
struct TriEdgeTrace {
  double phi, psi, dphi_m, n_m;
};

template <int P>
__device__ __forceinline__ void tri_edge_trace(const double *s_t, const TriLayout &L, int type, int f, int fk,
                                               const double *fphi, const double *fpsi, double ihl, double sgn,
                                               TriEdgeTrace *o) {
  constexpr int P1 = P + 1, NP = (P + 1) * (P + 2) / 2;
  const double *bev = s_t + L.bev() + fk * P1, *bet = s_t + L.bet() + fk * P1;
  const double *bn = s_t + L.bn() + (type * L.NQE + fk) * NP;
  double ph = 0.0, ps = 0.0, pt = 0.0, gp = 0.0, gs = 0.0;
#pragma unroll
  for (int m = 0; m < P1; ++m) {
    const int n = tri_edge_node(P, f, m);
    ph = fma(bev[m], fphi[n], ph);
    ps = fma(bev[m], fpsi[n], ps);
    pt = fma(bet[m], fpsi[n], pt);
  }
#pragma unroll
  for (int n = 0; n < NP; ++n) {
    gp = fma(bn[n], fphi[n], gp);
    gs = fma(bn[n], fpsi[n], gs);
  }
  const double st = pt * ihl;  // tangential derivative of psi
  const double g2 = gs * gs + st * st;
  o->phi = ph;
  o->psi = ps;
  o->dphi_m = sgn * gp;
  o->n_m = g2 < 1e-24 ? 0.0 : sgn * gs * rsqrt(g2);  // n = 0 where |grad psi| < 1e-12
}

// One stage: the right-hand side L = M^-1 R(win) at time *t0 + kstep dt + frac dt,
// written as L (KIN_RHS) or as one classical RK4 stage (KIN_K1..K4, the same
// updates as k_kin_stage; out may be w0, each node being read, then written,
// by the same thread).
template <int P>
__global__ void __launch_bounds__(TriGeom<P>::THREADS)
k_tri_stage(const KinParams kp, int mode, int kstep, double frac, const double *__restrict__ win,
            const double *w0, double *__restrict__ acc, double *out) {
  const double dt = __ldg(kp.dt);  // step size and stage time as in k_kin_stage
  const double tstep = kstep * dt, toff = frac * dt;
  using G = TriGeom<P>;
  constexpr TriLayout L = G::L;
  constexpr int NP = G::NP, NQ1 = G::NQ1, NQV = G::NQV, NQE = G::NQE, EPB = G::EPB;
  constexpr int NPT = NQV + NQE;
  __shared__ double s_t[L.size()];
  __shared__ double s_w[EPB][2][NP];
  __shared__ double s_nb[EPB][3][2][NP];
  __shared__ double s_cv[EPB][NQV][4];
  __shared__ double s_ce[EPB][NQE][4];
  __shared__ double s_R[EPB][2][NP];
  for (int i = threadIdx.x; i < L.size(); i += blockDim.x) s_t[i] = kp.ops[i];
  const double c = kin_time_factor(kp, (*kp.t0 + tstep) + toff);
  const int N = kp.N, ngroups = (kp.E + EPB - 1) / EPB;
  bool bad = false;

  for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int e0 = grp * EPB;
    __syncthreads();  // tables staged; the previous group's shared data consumed
    // 1. Own (slot 0) and neighbour (slots 1..3) nodal values.
    for (int it = threadIdx.x; it < EPB * 4 * NP; it += blockDim.x) {
      const int n = it % NP, slot = (it / NP) % 4, le = it / (4 * NP), e = e0 + le;
      double a = 0.0, b = 0.0;
      if (e < kp.E) {
        int f2, src = e;
        if (slot > 0) src = tri_neighbour(kp, e, slot - 1, &f2);
        if (in_bounds(kp.status, (long)src * NP + n, N)) {
          a = win[(long)src * NP + n];
          b = win[N + (long)src * NP + n];
        }
      }
      double *dst = slot == 0 ? s_w[le][0] : s_nb[le][slot - 1][0];
      dst[n] = a;
      dst[NP + n] = b;
    }
    __syncthreads();
    // 2. Volume points: coefficients of l_n, dl_n/dr, dl_n/ds (phi) and l_n (psi).
    for (int it = threadIdx.x; it < EPB * NQV; it += blockDim.x) {
      const int le = it / NQV, q = it % NQV, e = e0 + le;
      double cv[4] = {0.0, 0.0, 0.0, 0.0};
      if (e < kp.E) {
        const TriConst &g = kp.tc[e & 1];
        TriPoint o;
        tri_eval_point<NP, false>(kp, g, s_w[le][0], s_w[le][1], s_t + L.bv() + q * NP, s_t + L.brv() + q * NP,
                           s_t + L.bsv() + q * NP, &o);
        const long ov = (long)e * NPT + q;
        const double2 U = in_bounds(kp.status, ov, (long long)kp.E * NPT)
                              ? __ldg(reinterpret_cast<const double2 *>(kp.vel_tab) + ov)
                              : make_double2(0.0, 0.0);
        const double u = U.x * c, v = U.y * c;
        const double wq = s_t[L.wv() + q] * g.det;
        cv[0] = -wq * (u * o.gp[0] + v * o.gp[1]);
        cv[1] = -wq * (o.a1[0] * g.rx + o.a1[1] * g.ry);
        cv[2] = -wq * (o.a1[0] * g.sx + o.a1[1] * g.sy);
        cv[3] = -wq * (u * o.gs[0] + v * o.gs[1]);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) s_cv[le][q][k] = cv[k];
    }
    // 3. Edge points: transport and SIP fluxes, the symmetric term.  On each side: phi and psi
    //    from the p+1 edge nodes, the normal derivatives of phi and psi from all nodes (bn), the
    //    tangential derivative of psi from the edge nodes -- n . m = (d psi/dm) / |grad psi|.
    for (int it = threadIdx.x; it < EPB * NQE; it += blockDim.x) {
      const int le = it / NQE, fk = it % NQE, f = fk / NQ1, k = fk % NQ1, e = e0 + le;
      double ce[4] = {0.0, 0.0, 0.0, 0.0};
      if (e < kp.E) {
        int f2;
        const int e2 = tri_neighbour(kp, e, f, &f2);
        const int fk2 = f2 * NQ1 + (NQ1 - 1 - k);  // the same physical point, seen from the neighbour
        const TriConst &g = kp.tc[e & 1], &g2 = kp.tc[e2 & 1];
        TriEdgeTrace om, op;
        tri_edge_trace<P>(s_t, L, e & 1, f, fk, s_w[le][0], s_w[le][1], g.ihl[f], 1.0, &om);
        tri_edge_trace<P>(s_t, L, e2 & 1, f2, fk2, s_nb[le][f][0], s_nb[le][f][1], g2.ihl[f2], -1.0, &op);
        const double2 *vt = reinterpret_cast<const double2 *>(kp.vel_tab);
        const long vm = (long)e * NPT + NQV + fk, vp = (long)e2 * NPT + NQV + fk2;
        const long long nt = (long long)kp.E * NPT;
        const double2 U = in_bounds(kp.status, vm, nt) ? __ldg(vt + vm) : make_double2(0.0, 0.0);
        const double2 U2 = in_bounds(kp.status, vp, nt) ? __ldg(vt + vp) : make_double2(0.0, 0.0);
        const double m0 = g.m0[f], m1 = g.m1[f];
        const double unm = U.x * c * m0 + U.y * c * m1, unp = U2.x * c * m0 + U2.y * c * m1;
        const double lam = fmax(fabs(unm), fabs(unp));
        const double wf = s_t[L.we() + k] * g.hl[f];
        const double jump = op.phi - om.phi, hjs = 0.5 * (op.psi - om.psi);
        const double gn = 0.5 * (op.dphi_m + om.dphi_m);
        const double sharp = 0.5 * (op.phi * (1.0 - op.phi) * op.n_m + om.phi * (1.0 - om.phi) * om.n_m);
        const double ahat = kp.Gamma * (kp.eps * (gn + g.eta[f] * jump) - sharp);
        const double sym = 0.5 * kp.Gamma * kp.eps * jump;
        ce[0] = wf * ((lam - unm) * 0.5 * jump + ahat);  // x l_n (edge nodes)
        ce[1] = -wf * sym;                                // x d l_n / dm (all nodes)
        ce[3] = wf * (lam - unm) * hjs;                   // x l_n (edge nodes), psi
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) s_ce[le][fk][q] = ce[q];
    }
    __syncthreads();
    // 4. Weak-form sums R_n: volume points, the lifted symmetric term at every edge point, and
    //    the edge fluxes at the edges the node lies on.
    for (int it = threadIdx.x; it < EPB * NP; it += blockDim.x) {
      const int le = it / NP, n = it % NP;
      double rp = 0.0, rs = 0.0;
#pragma unroll 4
      for (int q = 0; q < NQV; ++q) {
        const double *cq = s_cv[le][q];
        const double b = s_t[L.bv() + q * NP + n];
        rp = fma(cq[0], b, rp);
        rp = fma(cq[1], s_t[L.brv() + q * NP + n], rp);
        rp = fma(cq[2], s_t[L.bsv() + q * NP + n], rp);
        rs = fma(cq[3], b, rs);
      }
      const double *bn = s_t + L.bn() + ((e0 + le) & 1) * NQE * NP;
#pragma unroll 4
      for (int q = 0; q < NQE; ++q) rp = fma(s_ce[le][q][1], bn[q * NP + n], rp);
      int ni = n, nj = 0;  // node (i, j) of index n
      while (ni > P - nj) {
        ni -= P + 1 - nj;
        ++nj;
      }
#pragma unroll 1
      for (int f = 0; f < 3; ++f) {
        const bool on = f == 0 ? nj == 0 : (f == 1 ? ni + nj == P : ni == 0);
        if (!on) continue;
        const int m = f == 0 ? ni : nj;  // its position along the edge (tri_edge_node)
#pragma unroll
        for (int k = 0; k < NQ1; ++k) {
          const double l = s_t[L.bev() + (f * NQ1 + k) * (P + 1) + m];
          rp = fma(s_ce[le][f * NQ1 + k][0], l, rp);
          rs = fma(s_ce[le][f * NQ1 + k][3], l, rs);
        }
      }
      s_R[le][0][n] = rp;
      s_R[le][1][n] = rs;
    }
    __syncthreads();
    // 5. L = M^-1 R / det and the stage update.
    for (int it = threadIdx.x; it < EPB * NP; it += blockDim.x) {
      const int le = it / NP, n = it % NP, e = e0 + le;
      if (e >= kp.E || !in_bounds(kp.status, (long)e * NP + n, N)) continue;
      const double idet = kp.tc[e & 1].idet;
#pragma unroll
      for (int vv = 0; vv < 2; ++vv) {
        double a = 0.0;
#pragma unroll
        for (int j = 0; j < NP; ++j) a = fma(s_t[L.minv() + n * NP + j], s_R[le][vv][j], a);
        const double Lv = a * idet;
        const long o = (long)vv * N + (long)e * NP + n;
        double r;
        if (mode == KIN_RHS) {
          r = Lv;
        } else {
          const double base = w0[o];
          if (mode == KIN_K1) {
            acc[o] = Lv;
            r = base + 0.5 * dt * Lv;
          } else if (mode == KIN_K2) {
            acc[o] += 2.0 * Lv;
            r = base + 0.5 * dt * Lv;
          } else if (mode == KIN_K3) {
            acc[o] += 2.0 * Lv;
            r = base + dt * Lv;
          } else {
            r = base + dt / 6.0 * (acc[o] + Lv);
          }
        }
        bad |= !isfinite(r);
        out[o] = r;
      }
    }
  }
  if (kp.check_finite && bad) atomicOr(kp.status, STATUS_NONFINITE);
}

struct TriKernels {
  cudaError_t (*stage)(const KinParams &, int mode, int kstep, double frac, const double *win, const double *w0,
                       double *acc, double *out, int grid, cudaStream_t);
  cudaError_t (*velocity_table)(const KinParams &, double *tab, cudaStream_t);
  const void *fn;  // the stage kernel, for the occupancy query
  int threads;
  int points;      // volume + edge points per triangle (rows of the velocity table)
};

template <int P>
cudaError_t launch_tri_stage(const KinParams &kp, int mode, int kstep, double frac, const double *win,
                             const double *w0, double *acc, double *out, int grid, cudaStream_t s) {
  k_tri_stage<P><<<grid, TriGeom<P>::THREADS, 0, s>>>(kp, mode, kstep, frac, win, w0, acc, out);
  return cudaGetLastError();
}

// Kernels of order p (1..4); false for other orders.
bool tri_kernels(int p, TriKernels *out);
// Triangles one CTA processes per pass (EPB of order p).
int tri_group(int p);
// Tables of order p in the TriLayout order, the normal derivatives for the two triangle types
// of constants tc; empty on failure.
std::vector<double> tri_tables(int p, const TriConst tc[2]);
// Constants of the two triangle types of cells hx x hy (penalty factor eta_tri = c_ip (p+1)(p+2)).
void tri_constants(double hx, double hy, double eta_tri, TriConst tc[2]);

}  // namespace dgpf
