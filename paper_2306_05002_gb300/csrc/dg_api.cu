// dg_api.cu -- host side of libdgpf: the C ABI declared in include/dgpf.h.
//
// Builds the operator tables (Gauss-Lobatto-Legendre nodes and weights, the
// Lagrange derivative matrix and the weak-form derivative Dhat = W^-1 D^T W of
// Sec. 3), owns the device workspace, launches the kernels of
// dg_kernels_fp64.cuh, captures SSP-RK3 step sequences in CUDA graphs, and
// runs the FP64 diagnostic reductions.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dg_common.cuh"
#include "dg_kernels_fp64.cuh"
#include "dg_kernels_fp32.cuh"
#include "dg_batch.cuh"
#include "dg_adjoint.cuh"
#include "dg_kin.cuh"
#include "dg_reinit.cuh"
#include "dg_tri.cuh"
#include "dg_host.h"
#include "dgpf.h"

namespace dgpf {
bool kernels_fp64_p1(int, bool, bool, KernelSet *);
bool kernels_fp64_p2(int, bool, bool, KernelSet *);
bool kernels_fp64_p3(int, bool, bool, KernelSet *);
bool kernels_fp64_p4(int, bool, bool, KernelSet *);
bool kernels_fp64_p5(int, bool, bool, KernelSet *);

bool kernels_fp32_p1(int, bool, bool, KernelSet32 *);
bool kernels_fp32_p2(int, bool, bool, KernelSet32 *);
bool kernels_fp32_p3(int, bool, bool, KernelSet32 *);
bool kernels_fp32_p4(int, bool, bool, KernelSet32 *);
bool kernels_fp32_p5(int, bool, bool, KernelSet32 *);

void batch_variants_p1(BatchVariant *);
void batch_variants_p2(BatchVariant *);
void batch_variants_p3(BatchVariant *);
void batch_variants_p4(BatchVariant *);
void batch_variants_p5(BatchVariant *);

bool batch_variants(int p, BatchVariant *out) {
  switch (p) {
    case 1: batch_variants_p1(out); return true;
    case 2: batch_variants_p2(out); return true;
    case 3: batch_variants_p3(out); return true;
    case 4: batch_variants_p4(out); return true;
    case 5: batch_variants_p5(out); return true;
    default: return false;
  }
}

bool kernels_fp32(int p, int dim, bool viscous, bool st, KernelSet32 *out) {
  switch (p) {
    case 1: return kernels_fp32_p1(dim, viscous, st, out);
    case 2: return kernels_fp32_p2(dim, viscous, st, out);
    case 3: return kernels_fp32_p3(dim, viscous, st, out);
    case 4: return kernels_fp32_p4(dim, viscous, st, out);
    case 5: return kernels_fp32_p5(dim, viscous, st, out);
    default: return false;
  }
}

// One value into device memory, in stream order (the step size of the captured dg_step graphs).
__global__ void k_set_double(double *dst, double v) { *dst = v; }

bool adj_kernels_p1(int, AdjKernels *);
bool adj_kernels_p2(int, AdjKernels *);
bool adj_kernels_p3(int, AdjKernels *);
bool adj_kernels_p4(int, AdjKernels *);
bool adj_kernels_p5(int, AdjKernels *);

bool adj_kernels(int p, int dim, AdjKernels *out) {
  switch (p) {
    case 1: return adj_kernels_p1(dim, out);
    case 2: return adj_kernels_p2(dim, out);
    case 3: return adj_kernels_p3(dim, out);
    case 4: return adj_kernels_p4(dim, out);
    case 5: return adj_kernels_p5(dim, out);
    default: return false;
  }
}

bool kernels_fp64(int p, int dim, bool viscous, bool st, KernelSet *out) {
  switch (p) {
    case 1: return kernels_fp64_p1(dim, viscous, st, out);
    case 2: return kernels_fp64_p2(dim, viscous, st, out);
    case 3: return kernels_fp64_p3(dim, viscous, st, out);
    case 4: return kernels_fp64_p4(dim, viscous, st, out);
    case 5: return kernels_fp64_p5(dim, viscous, st, out);
    default: return false;
  }
}

// ---------------------------------------------------------------------------
// Diagnostics: deterministic two-pass FP64 reduction.
// ---------------------------------------------------------------------------
constexpr int DIAG_THREADS = 256;
constexpr int DIAG_N = 16;

__device__ __forceinline__ void diag_combine(double *a, const double *b) {
  for (int q = 0; q < 7; ++q) a[q] += b[q];
  a[7] = fmin(a[7], b[7]);  a[8] = fmax(a[8], b[8]);
  a[9] = fmin(a[9], b[9]);  a[10] = fmax(a[10], b[10]);
  a[11] = fmin(a[11], b[11]); a[12] = fmax(a[12], b[12]);
  a[13] = fmin(a[13], b[13]); a[14] = fmax(a[14], b[14]);
  a[15] += b[15];
}

__device__ __forceinline__ void diag_identity(double *a) {
  for (int q = 0; q < 7; ++q) a[q] = 0.0;
  for (int q = 7; q < 15; q += 2) { a[q] = INFINITY; a[q + 1] = -INFINITY; }
  a[15] = 0.0;
}

__device__ void diag_block_reduce(double (*sh)[DIAG_N], double *mine, double *dst) {
  for (int q = 0; q < DIAG_N; ++q) sh[threadIdx.x][q] = mine[q];
  __syncthreads();
  for (int s = DIAG_THREADS / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) diag_combine(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < DIAG_N; ++q) dst[q] = sh[0][q];
}

__global__ void __launch_bounds__(DIAG_THREADS)
k_diag_partial(const Params prm, int Np, int P1, int dim, double J, const double *__restrict__ w,
               double *__restrict__ part) {
  __shared__ double sh[DIAG_THREADS][DIAG_N];
  double acc[DIAG_N];
  diag_identity(acc);
  const double *wt = prm.ops + OpsLayout{P1, Np}.wt();
  for (long n = blockIdx.x * (long)DIAG_THREADS + threadIdx.x; n < prm.N; n += (long)gridDim.x * DIAG_THREADS) {
    const int a = (int)(n % Np);
    const double wJ = (dim == 2 ? wt[a % P1] * wt[a / P1] : wt[a]) * J;
    double q[NV];
    for (int v = 0; v < NV; ++v) {
      q[v] = w[(long)v * prm.N + n];
      acc[v] += wJ * q[v];
      if (!isfinite(q[v])) acc[15] += 1.0;
    }
    const double rho = q[M1] + q[M2];
    double Cm, den;
    const double P = sg_pressure(prm, q[PHI], rho, q[RU], q[RV], q[RE], &Cm, &den);
    const double u = q[RU] / rho, v = q[RV] / rho;
    acc[7] = fmin(acc[7], q[PHI]);  acc[8] = fmax(acc[8], q[PHI]);
    acc[9] = fmin(acc[9], P);       acc[10] = fmax(acc[10], P);
    acc[11] = fmin(acc[11], u);     acc[12] = fmax(acc[12], u);
    acc[13] = fmin(acc[13], v);     acc[14] = fmax(acc[14], v);
  }
  diag_block_reduce(sh, acc, part + (long)blockIdx.x * DIAG_N);
}

__global__ void __launch_bounds__(DIAG_THREADS)
k_diag_final(int nparts, const double *__restrict__ part, double *__restrict__ out) {
  __shared__ double sh[DIAG_THREADS][DIAG_N];
  double acc[DIAG_N];
  diag_identity(acc);
  for (int b = threadIdx.x; b < nparts; b += DIAG_THREADS) diag_combine(acc, part + (long)b * DIAG_N);
  diag_block_reduce(sh, acc, out);
}

}  // namespace dgpf

using namespace dgpf;

// ---------------------------------------------------------------------------
// Operator tables (host)
// ---------------------------------------------------------------------------
namespace {

// Vector forms of the shared table builders (dg_host.h).
void gll_nodes(int p, std::vector<double> &x, std::vector<double> &w) {
  x.assign(p + 1, 0.0);
  w.assign(p + 1, 0.0);
  gll_nodes_into(p, x.data(), w.data());
}

thread_local std::string g_create_error = "no error";

#ifdef DG_CHECK
// Bounds failures seen by dg_status_read or found latched by dg_destroy (bounds-checked build).
std::atomic<long long> g_bounds_failures{0};
#endif

}  // namespace

// A batch of independent problems advanced together (dg_batch_create).
struct BatchGroup {
  int p = 0;
  std::vector<int> probs;          // problem indices of this order
  BatchProb *d_probs = nullptr;    // descriptors, in the order of `probs`
  BatchVariant var[NVAR] = {};     // tile variants of this order
  int *d_block0[NVAR] = {};        // first block of each problem, per variant
  int nblocks[NVAR] = {};
  int best = -1;                   // chosen variant (-1: not tuned yet)
  double ms[NVAR] = {};            // tuning times (volume + two fused launches)
  cudaStream_t stream = nullptr;   // capture branch of this group
  cudaEvent_t done = nullptr;      // joins the branch back at the end of a captured sequence
};

struct BatchData {
  int n = 0;
  std::vector<BatchProb> h;        // descriptor of every problem (host copy)
  std::vector<int> group_of, slot_of;
  std::vector<BatchGroup> groups;
  std::vector<size_t> len;         // state length of every problem
  void *d_pool = nullptr;          // every FP32 buffer and table of the batch
  cudaEvent_t fork = nullptr;      // starts the per-group branches of a captured sequence
};

struct dg_ctx {
  BatchData *batch = nullptr;
  dg_mesh mesh;
  int p;
  dg_eos eos;
  double Gamma, eps;
  dg_opts opts;
  int dim, P1, Np, E, N, NFK;
  size_t len;
  double hx, hy, J;
  Params prm;
  KernelSet ks;
  KernelSet32 ks32;
  ParamsF pf;
  int prec = DG_FP64;
  AdjKernels adj{};
  bool has_adj = false;
  double *d_trbar = nullptr, *d_lam1 = nullptr, *d_lam2 = nullptr;
  // FP32-bulk: step start (hi and lo parts, double-buffered) and the two inner stage increments
  float *d_hi32[2] = {}, *d_lo32[2] = {}, *d_dd32[2] = {};
  float *d_opsf = nullptr, *d_rvol32 = nullptr,
        *d_trace32 = nullptr, *d_rvol32b = nullptr, *d_trace32b = nullptr;
  double *d_ops = nullptr, *d_w1 = nullptr, *d_w2 = nullptr, *d_rvol = nullptr, *d_trace = nullptr;
  double *d_hstate = nullptr;  // device copy of a host state (dg_step_host), allocated on first use
  double *d_copy64 = nullptr;  // FP32-bulk single steps on a page-locked host state (enqueue_steps32)
  // kinematic mode (dg_kin_create); tri: triangles (one fused kernel per stage)
  bool kin = false, tri = false;
  KinParams kp{};
  KinKernels kk{};
  TriKernels tk{};
  int tri_grid = 0;
  double *d_kacc = nullptr, *d_kwsA = nullptr, *d_kwsB = nullptr;
  double *d_kt0 = nullptr, *d_kxi = nullptr, *d_ktv = nullptr;
  // level-set re-initialisation workspace (dg_reinit), allocated on first use
  double *d_riS = nullptr, *d_ri1 = nullptr, *d_ri2 = nullptr, *d_rirvol = nullptr, *d_ritr = nullptr;
  double *d_part = nullptr, *d_diag = nullptr;
  unsigned *d_status = nullptr;
  int nparts = 0;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t g1 = nullptr, gk = nullptr;  // dg_batch_step, dg_kin_step
  // dg_step: the captured step graphs of the two state arrays used most recently (one step,
  // GRAPH_UNROLL steps, and for FP32-bulk the remainders of 2..7 steps, captured on first use), so
  // that a caller alternating two buffers captures once per buffer
  struct StepGraphs {
    const double *w = nullptr;
    cudaGraphExec_t g1 = nullptr, gk = nullptr;
    cudaGraphExec_t grem[8] = {};
    unsigned long long used = 0;
  } sg[2];
  unsigned long long sg_clock = 0;
  // dg_adjoint_segment: captured segment sweeps, keyed by (steps, dt, states, tapes, lam)
  struct SegGraph {
    cudaGraphExec_t exec = nullptr;
    int m = 0;
    double dt = 0.0;
    const double *states = nullptr, *tapes = nullptr, *lam = nullptr;
  } seg[2];
  const double *g_w = nullptr;
  double *d_dt = nullptr;      // the step size the captured dg_step / dg_kin_step graphs read
  double dt_set = 0.0;         // the value last written there (0: none)
  std::string err = "no error";
};

static const int GRAPH_UNROLL = 8;
static_assert(GRAPH_UNROLL <= (int)(sizeof(dg_ctx::StepGraphs::grem) / sizeof(cudaGraphExec_t)),
              "remainder graph slots");

static dg_status fail(dg_ctx *c, dg_status s, const std::string &msg) {
  if (c) c->err = msg;
  else g_create_error = msg;
  return s;
}

static dg_status cuda_fail(dg_ctx *c, cudaError_t e, const char *what) {
  return fail(c, DG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static void free_step_graphs(dg_ctx::StepGraphs *G) {
  if (G->g1) cudaGraphExecDestroy(G->g1);
  if (G->gk) cudaGraphExecDestroy(G->gk);
  for (auto &g : G->grem)
    if (g) cudaGraphExecDestroy(g);
  *G = dg_ctx::StepGraphs{};
}

static void free_graphs(dg_ctx *c) {
  if (c->g1) cudaGraphExecDestroy(c->g1);
  if (c->gk) cudaGraphExecDestroy(c->gk);
  c->g1 = c->gk = nullptr;
  c->g_w = nullptr;
  for (auto &G : c->sg) free_step_graphs(&G);
}

static void free_seg_graphs(dg_ctx *c) {
  for (auto &g : c->seg) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = dg_ctx::SegGraph{};
  }
}

static void free_ctx(dg_ctx *c) {
  if (!c) return;
  free_graphs(c);
  free_seg_graphs(c);
  if (c->batch) {
    for (auto &g : c->batch->groups) {
      cudaFree(g.d_probs);
      for (auto *p0 : g.d_block0) cudaFree(p0);
      if (g.stream) cudaStreamDestroy(g.stream);
      if (g.done) cudaEventDestroy(g.done);
    }
    if (c->batch->fork) cudaEventDestroy(c->batch->fork);
    cudaFree(c->batch->d_pool);
    delete c->batch;
  }
  cudaFree(c->d_ops);
  cudaFree(c->d_hstate);
  cudaFree(c->d_copy64);
  for (double *q : {c->d_kacc, c->d_kwsA, c->d_kwsB, c->d_kt0, c->d_kxi, c->d_ktv}) cudaFree(q);
  for (double *q : {c->d_riS, c->d_ri1, c->d_ri2, c->d_rirvol, c->d_ritr}) cudaFree(q);
  cudaFree(c->d_w1);
  cudaFree(c->d_w2);
  cudaFree(c->d_rvol);
  cudaFree(c->d_trace);
  cudaFree(c->d_part);
  cudaFree(c->d_diag);
  cudaFree(c->d_status);
  cudaFree(c->d_dt);
  cudaFree(c->d_trbar);
  cudaFree(c->d_lam1);
  cudaFree(c->d_lam2);
  cudaFree(c->d_opsf);
  for (int k = 0; k < 2; ++k) {
    cudaFree(c->d_hi32[k]);
    cudaFree(c->d_lo32[k]);
    cudaFree(c->d_dd32[k]);
  }
  cudaFree(c->d_rvol32);
  cudaFree(c->d_trace32);
  cudaFree(c->d_rvol32b);
  cudaFree(c->d_trace32b);
  if (c->cap) cudaStreamDestroy(c->cap);
  delete c;
}

// Operator table (OpsLayout) for one element size.
static std::vector<double> build_ops(int dim, int p, double hx, double hy) {
  const int P1 = p + 1;
  std::vector<double> ops(OpsLayout{P1, dim == 2 ? P1 * P1 : P1}.size(), 0.0);
  build_ops_into(dim, p, hx, hy, ops.data());
  return ops;
}

extern "C" dg_status dg_create(const dg_mesh *mesh, int p, const dg_eos *eos, double Gamma, double eps,
                               const dg_opts *opts, dg_ctx **out) {
  if (!out) return fail(nullptr, DG_ERR_ARG, "dg_create: out is NULL");
  *out = nullptr;
  dg_status code;
  if (const char *why = check_problem(mesh, p, eos, Gamma, eps, &code))
    return fail(nullptr, code, std::string("dg_create: ") + why);
  const dg_opts o = normalised_opts(opts);
  if (o.prec != DG_FP64 && o.prec != DG_FP32_BULK)
    return fail(nullptr, DG_ERR_ARG, "dg_create: precision must be DG_FP64 or DG_FP32_BULK");
  if (o.grad_lift != 0 && o.grad_lift != 1) return fail(nullptr, DG_ERR_ARG, "dg_create: grad_lift must be 0 or 1");
  if (o.grad_lift && o.prec != DG_FP64)
    return fail(nullptr, DG_ERR_UNSUPPORTED, "dg_create: lifted gradients (grad_lift) are built by the FP64 kernels");
  const long long E = (long long)mesh->nx * mesh->ny;
  const int P1 = p + 1;
  const int Np = mesh->dim == 2 ? P1 * P1 : P1;

  dg_ctx *c = new (std::nothrow) dg_ctx();
  if (!c) return fail(nullptr, DG_ERR_OOM, "dg_create: host allocation failed");
  c->mesh = *mesh;
  c->p = p;
  c->eos = *eos;
  c->Gamma = Gamma;
  c->eps = eps;
  c->opts = o;
  c->dim = mesh->dim;
  c->P1 = P1;
  c->Np = Np;
  c->E = (int)E;
  c->N = (int)(E * Np);
  c->NFK = 2 * c->dim * (c->dim == 2 ? P1 : 1);
  c->len = (size_t)NV * c->N;
  c->hx = (mesh->x1 - mesh->x0) / mesh->nx;
  c->hy = c->dim == 2 ? (mesh->y1 - mesh->y0) / mesh->ny : 1.0;
  c->J = c->dim == 2 ? 0.25 * c->hx * c->hy : 0.5 * c->hx;

  c->prec = o.prec;
  if (!kernels_fp64(p, c->dim, o.viscous != 0, o.surface_tension != 0, &c->ks) ||
      !kernels_fp32(p, c->dim, o.viscous != 0, o.surface_tension != 0, &c->ks32)) {
    free_ctx(c);
    return fail(nullptr, DG_ERR_UNSUPPORTED, "dg_create: viscous/surface terms need dim = 2");
  }

  // The discrete adjoint covers the FP64 inviscid equations without surface tension.
  bool pressure_bc = false;
  for (int f = 0; f < 4; ++f) pressure_bc |= mesh->bc[f] == DG_BC_PRESSURE;
  c->has_adj = c->prec == DG_FP64 && !o.viscous && !o.surface_tension && !pressure_bc && !o.grad_lift &&
               adj_kernels(p, c->dim, &c->adj);
  const std::vector<double> ops = build_ops(c->dim, p, c->hx, c->hy);
  c->prm = make_params(mesh, p, eos, Gamma, eps, o, c->hx, c->hy);
  Params &q = c->prm;

  cudaError_t e = cudaSuccess;
  const bool f64 = c->prec == DG_FP64;
  const size_t sbytes = c->len * sizeof(double);
  const size_t tbytes = (size_t)c->ks.nt * c->E * c->NFK * sizeof(double);
  c->nparts = std::min(1024, (c->N + DIAG_THREADS - 1) / DIAG_THREADS);
  c->pf = to_float(c->prm);
  std::vector<float> opsf(ops.begin(), ops.end());
  auto alloc32 = [&](float **ptr, size_t n) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, n * sizeof(float));
    return e == cudaSuccess;
  };
  if (!f64) {
    const size_t n32 = (size_t)SW32 * c->N;  // one padded record per node (inviscid kernels)
    const size_t t32 = (size_t)TRW32 * c->E * c->NFK;  // one padded record per face node
    alloc32(&c->d_opsf, opsf.size()) && alloc32(&c->d_hi32[0], n32) && alloc32(&c->d_hi32[1], n32) &&
        alloc32(&c->d_lo32[0], n32) && alloc32(&c->d_lo32[1], n32) && alloc32(&c->d_dd32[0], n32) &&
        alloc32(&c->d_dd32[1], n32) && alloc32(&c->d_rvol32, n32) && alloc32(&c->d_trace32, t32) &&
        alloc32(&c->d_rvol32b, n32) && alloc32(&c->d_trace32b, t32);
  }
  if (e != cudaSuccess || (e = cudaMalloc(&c->d_ops, ops.size() * sizeof(double))) != cudaSuccess ||
      (f64 && ((e = cudaMalloc(&c->d_w1, sbytes)) != cudaSuccess || (e = cudaMalloc(&c->d_w2, sbytes)) != cudaSuccess ||
               (e = cudaMalloc(&c->d_rvol, sbytes)) != cudaSuccess ||
               (e = cudaMalloc(&c->d_trace, tbytes)) != cudaSuccess)) ||
      (e = cudaMalloc(&c->d_part, (size_t)c->nparts * DIAG_N * sizeof(double))) != cudaSuccess ||
      (c->has_adj && ((e = cudaMalloc(&c->d_trbar, (size_t)NT_INVISCID * c->E * c->NFK * sizeof(double))) !=
                          cudaSuccess ||
                      (e = cudaMalloc(&c->d_lam1, sbytes)) != cudaSuccess ||
                      (e = cudaMalloc(&c->d_lam2, sbytes)) != cudaSuccess)) ||
      (e = cudaMalloc(&c->d_diag, DIAG_N * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&c->d_dt, sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&c->d_status, sizeof(unsigned))) != cudaSuccess) {
    free_ctx(c);
    cudaGetLastError();
    return fail(nullptr, e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA,
                std::string("dg_create: device allocation failed: ") + cudaGetErrorString(e));
  }
  if ((e = cudaMemcpy(c->d_ops, ops.data(), ops.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (!f64 && (e = cudaMemcpy(c->d_opsf, opsf.data(), opsf.size() * sizeof(float), cudaMemcpyHostToDevice)) !=
                   cudaSuccess) ||
      (e = cudaMemset(c->d_status, 0, sizeof(unsigned))) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking)) != cudaSuccess) {
    free_ctx(c);
    return fail(nullptr, DG_ERR_CUDA, std::string("dg_create: ") + cudaGetErrorString(e));
  }
  q.ops = c->d_ops;
  q.status = c->d_status;
  *out = c;
  return DG_OK;
}

extern "C" void dg_destroy(dg_ctx *c) {
  if (!c) return;
  cudaDeviceSynchronize();
#ifdef DG_CHECK
  // a bounds failure nobody read is counted before the word goes away
  unsigned h = 0;
  if (c->d_status && cudaMemcpy(&h, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost) == cudaSuccess &&
      (h & STATUS_BOUNDS))
    ++g_bounds_failures;
#endif
  free_ctx(c);
}

// Self-test of the bounds-checked build: the FP64 volume kernel of a 2 x 2, p = 2 periodic problem
// runs with a node count one short of the mesh's.  Every array keeps its true size, so no access
// leaves its allocation (the field offsets v (N - 1) + n stay below 7 N); only the last node's
// index fails its check, which must latch STATUS_BOUNDS and skip that node.
extern "C" int dg_check_selftest(void *stream) {
#ifndef DG_CHECK
  (void)stream;
  return DG_ERR_UNSUPPORTED;
#else
  dg_mesh m{};
  m.dim = 2;
  m.nx = m.ny = 2;
  m.x1 = m.y1 = 1.0;
  dg_eos eos{};
  eos.gamma[0] = 1.4;
  eos.gamma[1] = 4.4;
  eos.pinf[1] = 6e8;
  eos.rho0[0] = 1.0;
  eos.rho0[1] = 1000.0;
  dg_ctx *c = nullptr;
  if (dg_create(&m, 2, &eos, 1.0, 0.1, nullptr, &c) != DG_OK) return DG_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  // air at rest at P = 1e5 (phi = 1, m1 = 1, rho E = P / (gamma - 1))
  std::vector<double> h(c->len, 0.0);
  const size_t N = (size_t)c->N;
  for (size_t n = 0; n < N; ++n) {
    h[PHI * N + n] = 1.0;
    h[M1 * N + n] = 1.0;
    h[RE * N + n] = 1e5 / 0.4;
  }
  Params q = c->prm;
  q.N -= 1;
  q.check_finite = 0;
  unsigned word = 0;
  cudaError_t e = cudaMemcpyAsync(c->d_w1, h.data(), c->len * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = c->ks.volume(q, c->d_w1, c->d_rvol, c->d_trace, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&word, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), s);  // planted: not a failure
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dg_destroy(c);
  if (e != cudaSuccess) return DG_ERR_CUDA;
  return (word & STATUS_BOUNDS) ? 1 : 0;
#endif
}

extern "C" int dg_check_build(long long *failures) {
#ifdef DG_CHECK
  if (failures) *failures = g_bounds_failures.load();
  return 1;
#else
  if (failures) *failures = 0;
  return 0;
#endif
}

extern "C" size_t dg_state_len(const dg_ctx *c) { return c ? c->len : 0; }

extern "C" const char *dg_last_error(const dg_ctx *c) { return c ? c->err.c_str() : g_create_error.c_str(); }

static dg_status run_stage(dg_ctx *c, int mode, double dt, const double *w0, const double *ws, double *out,
                           cudaStream_t s, const Params *prm = nullptr) {
  const Params &q = prm ? *prm : c->prm;
  cudaError_t e = c->ks.volume(q, ws, c->d_rvol, c->d_trace, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "volume kernel launch");
  e = c->ks.surface(q, mode, dt, w0, ws, c->d_rvol, c->d_trace, out, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "surface kernel launch");
  return DG_OK;
}

// The FP32-bulk right-hand side of the FP64 state w64: the volume kernel splits
// the state into the internal hi part (the lo part is not needed) and the
// surface kernel writes L in FP64.
static dg_status rhs32(dg_ctx *c, const double *w64, double *L, cudaStream_t s) {
  cudaError_t e = c->ks32.volume(c->prm, c->pf, c->d_opsf, nullptr, c->d_rvol32, c->d_trace32, w64, c->d_hi32[0],
                                 nullptr, nullptr, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "volume kernel launch");
  const StageIO io{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, L, nullptr};
  e = c->ks32.surface(c->prm, c->pf, c->d_opsf, MODE_RHS, 0.f, io, c->d_rvol32, c->d_trace32, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "surface kernel launch");
  return DG_OK;
}

extern "C" dg_status dg_rhs(dg_ctx *c, const double *w, double *L, void *stream) {
  if (!c) return DG_ERR_ARG;
  if (c->batch || c->kin) return fail(c, DG_ERR_ARG, "dg_rhs: batch or kinematic context");
  if (!w || !L) return fail(c, DG_ERR_ARG, "dg_rhs: null array");
  if (w == L) return fail(c, DG_ERR_ARG, "dg_rhs: w and L must not overlap");
  cudaStream_t s = (cudaStream_t)stream;
  if (c->prec == DG_FP64) return run_stage(c, MODE_RHS, 0.0, w, w, L, s);
  return rhs32(c, w, L, s);
}

// One SSP-RK3 step (Shu-Osher): w1 = w + dt L(w); w2 = 3/4 w + 1/4 (w1 + dt L(w1));
// w <- 1/3 w + 2/3 (w2 + dt L(w2)).  The last stage writes w in place (each
// node's w0 value is read by the thread that overwrites it).
// The captured sequences read dt from c->d_dt at run time, so a new dt needs no new capture.
static dg_status enqueue_step(dg_ctx *c, double *w, double dt, cudaStream_t s) {
  dg_status r;
  Params q = c->prm;
  q.dt_dev = c->d_dt;
  if ((r = run_stage(c, MODE_S1, dt, w, w, c->d_w1, s, &q)) != DG_OK) return r;
  if ((r = run_stage(c, MODE_S2, dt, w, c->d_w1, c->d_w2, s, &q)) != DG_OK) return r;
  return run_stage(c, MODE_S3, dt, w, c->d_w2, w, s, &q);
}

// `steps` FP32-bulk steps with the fused stage kernel: 1 + 3 steps launches.
// The volume part of the first stage reads the FP64 state and splits it into
// the internal step start (hi, lo); the last stage writes hi + lo back.  In
// between the state stays in FP32 pairs, whose sum keeps ~48 bits: a call of
// several steps differs from as many single-step calls (which add the last
// increment to the FP64 state in FP64) only by that rounding of each step's
// sum, far below the FP32 rounding of the increments themselves.
// Stage 1 writes the increment d1 into D[0], stage 2 reads it and writes d2
// into D[1], stage 3 adds 2 (d2 + dt L) / 3 to the step start in float-float
// and writes the new step start into the other buffer of each pair (H, Lo),
// so that no launch writes an array it also reads; the volume part and the
// traces alternate between the two buffers of their pairs.
// copy64 != NULL (a single step on a state in host memory): the first launch also copies the
// FP64 state it reads into copy64 (device memory), and the last adds its increment to that copy,
// so that the state crosses the host link once each way.
static dg_status enqueue_steps32(dg_ctx *c, double *w, float dt, int steps, cudaStream_t s,
                                 double *copy64 = nullptr) {
  float *const *H = c->d_hi32, *const *Lo = c->d_lo32, *const *D = c->d_dd32;
  float *rv[2] = {c->d_rvol32, c->d_rvol32b}, *tr[2] = {c->d_trace32, c->d_trace32b};
  int t = 0, a = 0;
  if (steps != 1) copy64 = nullptr;
  // a single step adds its last increment to the FP64 state itself: no lo part is needed
  cudaError_t e = c->ks32.volume(c->prm, c->pf, c->d_opsf, nullptr, rv[t], tr[t], w, H[a], steps > 1 ? Lo[a] : nullptr,
                                 copy64, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "volume kernel launch");
  for (int k = 0; k < steps; ++k) {
    const bool last = k == steps - 1;
    const StageIO io[3] = {
        {H[a], nullptr, nullptr, D[0], nullptr, nullptr, nullptr, nullptr, c->d_dt},
        {H[a], nullptr, D[0], D[1], nullptr, nullptr, nullptr, nullptr, c->d_dt},
        {H[a], Lo[a], D[1], nullptr, last ? nullptr : H[a ^ 1], last ? nullptr : Lo[a ^ 1], last ? w : nullptr,
         steps == 1 ? (copy64 ? copy64 : w) : nullptr, c->d_dt}};
    const int mode[3] = {MODE_S1, MODE_S2, MODE_S3};
    for (int st = 0; st < 3; ++st) {
      if (st == 2 && last) {
        e = c->ks32.surface(c->prm, c->pf, c->d_opsf, MODE_S3, dt, io[2], rv[t], tr[t], s);
        if (e != cudaSuccess) return cuda_fail(c, e, "surface kernel launch");
        break;
      }
      e = c->ks32.surfvol(c->prm, c->pf, c->d_opsf, mode[st], dt, io[st], rv[t], tr[t], rv[t ^ 1], tr[t ^ 1], s);
      if (e != cudaSuccess) return cuda_fail(c, e, "fused stage kernel launch");
      t ^= 1;
    }
    a ^= 1;  // the new step start is in the other buffer of each pair
  }
  return DG_OK;
}

static dg_status capture(dg_ctx *c, double *w, double dt, int steps, cudaGraphExec_t *exec) {
  double *copy64 = nullptr;
  if (c->prec != DG_FP64 && steps == 1) {
    // a state in page-locked host memory, read and written in place over the host link
    cudaPointerAttributes at{};
    const bool host = cudaPointerGetAttributes(&at, w) == cudaSuccess && at.type == cudaMemoryTypeHost;
    cudaGetLastError();
    if (host) {
      if (!c->d_copy64) {
        cudaError_t e = cudaMalloc(&c->d_copy64, c->len * sizeof(double));
        if (e != cudaSuccess) {
          c->d_copy64 = nullptr;
          cudaGetLastError();
          return fail(c, e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA,
                      std::string("dg_step: device copy of a host state: ") + cudaGetErrorString(e));
        }
      }
      copy64 = c->d_copy64;
    }
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_step: begin capture");
  dg_status r = DG_OK;
  if (c->prec != DG_FP64) r = enqueue_steps32(c, w, (float)dt, steps, c->cap, copy64);
  else
    for (int s = 0; s < steps && r == DG_OK; ++s) r = enqueue_step(c, w, dt, c->cap);
  e = cudaStreamEndCapture(c->cap, &g);
  if (r != DG_OK) {
    if (g) cudaGraphDestroy(g);
    return r;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_step: end capture");
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_step: instantiate");
  return DG_OK;
}

extern "C" dg_status dg_step(dg_ctx *c, double *w, double dt, int nsteps, void *stream) {
  if (!c) return DG_ERR_ARG;
  if (c->batch || c->kin) return fail(c, DG_ERR_ARG, "dg_step: batch or kinematic context");
  if (!w) return fail(c, DG_ERR_ARG, "dg_step: null state");
  if (!(dt > 0.0) || nsteps < 0) return fail(c, DG_ERR_ARG, "dg_step: need dt > 0 and nsteps >= 0");
  if (nsteps == 0) return DG_OK;
  dg_ctx::StepGraphs *G = nullptr;
  for (auto &x : c->sg)
    if (x.g1 && x.w == w) G = &x;
  if (!G) {  // capture for this state array, in a free slot or over the least recently used one
    G = !c->sg[0].g1 ? &c->sg[0] : !c->sg[1].g1 ? &c->sg[1] : c->sg[0].used <= c->sg[1].used ? &c->sg[0] : &c->sg[1];
    free_step_graphs(G);
    dg_status r;
    if ((r = capture(c, w, dt, 1, &G->g1)) != DG_OK || (r = capture(c, w, dt, GRAPH_UNROLL, &G->gk)) != DG_OK) {
      free_step_graphs(G);
      return r;
    }
    G->w = w;
  }
  G->used = ++c->sg_clock;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (dt != c->dt_set) {  // the graphs read the step size from device memory
    k_set_double<<<1, 1, 0, s>>>(c->d_dt, dt);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "dg_step: set dt");
    c->dt_set = dt;
  }
  for (int k = 0; k < nsteps / GRAPH_UNROLL; ++k)
    if ((e = cudaGraphLaunch(G->gk, s)) != cudaSuccess) return cuda_fail(c, e, "dg_step: graph launch");
  const int rem = nsteps % GRAPH_UNROLL;
  if (c->prec != DG_FP64 && rem > 1) {  // FP32-bulk: the remainder as one graph (fewer launches)
    if (!G->grem[rem]) {
      dg_status r;
      if ((r = capture(c, w, dt, rem, &G->grem[rem])) != DG_OK) return r;
    }
    if ((e = cudaGraphLaunch(G->grem[rem], s)) != cudaSuccess) return cuda_fail(c, e, "dg_step: graph launch");
    return DG_OK;
  }
  for (int k = 0; k < rem; ++k)
    if ((e = cudaGraphLaunch(G->g1, s)) != cudaSuccess) return cuda_fail(c, e, "dg_step: graph launch");
  return DG_OK;
}

extern "C" dg_status dg_step_host(dg_ctx *c, double *w_host, double dt, int nsteps, void *stream) {
  if (!c) return DG_ERR_ARG;
  if (c->batch || c->kin) return fail(c, DG_ERR_ARG, "dg_step_host: batch or kinematic context");
  if (!w_host) return fail(c, DG_ERR_ARG, "dg_step_host: null state");
  if (!(dt > 0.0) || nsteps < 0) return fail(c, DG_ERR_ARG, "dg_step_host: need dt > 0 and nsteps >= 0");
  if (nsteps == 0) return DG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  // FP32-bulk reads the FP64 state once per call (first stage) and writes it
  // once (last stage).  When w_host is page-locked and mapped into the device
  // address space, those two kernels access it in place over the host link
  // (NVLink-C2C on GB300), with no staging copies.
  if (c->prec != DG_FP64) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, w_host) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer) {
      const dg_status r = dg_step(c, static_cast<double *>(at.devicePointer), dt, nsteps, stream);
      if (r != DG_OK) return r;
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(c, e, "dg_step_host: sync");
      return DG_OK;
    }
    cudaGetLastError();
  }
  if (!c->d_hstate && (e = cudaMalloc(&c->d_hstate, c->len * sizeof(double))) != cudaSuccess) {
    c->d_hstate = nullptr;
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA,
                std::string("dg_step_host: staging buffer: ") + cudaGetErrorString(e));
  }
  const size_t bytes = c->len * sizeof(double);
  if ((e = cudaMemcpyAsync(c->d_hstate, w_host, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_fail(c, e, "dg_step_host: copy to device");
  const dg_status r = dg_step(c, c->d_hstate, dt, nsteps, stream);
  if (r != DG_OK) {
    cudaStreamSynchronize(s);
    return r;
  }
  if ((e = cudaMemcpyAsync(w_host, c->d_hstate, bytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(c, e, "dg_step_host: copy to host");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(c, e, "dg_step_host: sync");
  return DG_OK;
}

extern "C" dg_status dg_diag(dg_ctx *c, const double *w, double *out, void *stream) {
  if (!c) return DG_ERR_ARG;
  if (c->batch || c->kin) return fail(c, DG_ERR_ARG, "dg_diag: batch or kinematic context");
  if (!w || !out) return fail(c, DG_ERR_ARG, "dg_diag: null array");
  cudaStream_t s = (cudaStream_t)stream;
  k_diag_partial<<<c->nparts, DIAG_THREADS, 0, s>>>(c->prm, c->Np, c->P1, c->dim, c->J, w, c->d_part);
  k_diag_final<<<1, DIAG_THREADS, 0, s>>>(c->nparts, c->d_part, c->d_diag);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_diag: launch");
  if ((e = cudaMemcpyAsync(out, c->d_diag, DIAG_N * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(c, e, "dg_diag: copy");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(c, e, "dg_diag: sync");
  return DG_OK;
}

extern "C" dg_status dg_status_read(dg_ctx *c, void *stream) {
  if (!c) return DG_ERR_ARG;
  if (!c->d_status) return DG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_status_read");
  if (h & STATUS_BOUNDS) {  // only the bounds-checked build sets it: a library bug, reported first
#ifdef DG_CHECK
    ++g_bounds_failures;
#endif
    return fail(c, DG_ERR_BOUNDS, "a kernel index left its array (bounds-checked build)");
  }
  // a non-physical state is reported first: it is the cause of the non-finite values it produces
  if (h & STATUS_NONPHYSICAL)
    return fail(c, DG_ERR_NONPHYSICAL, "non-physical state on the device (rho <= 0 or P + Pinf <= 0)");
  if (h & STATUS_NONFINITE) return fail(c, DG_ERR_NONFINITE, "non-finite value produced on the device");
  return DG_OK;
}

extern "C" int dg_time_kernels(dg_ctx *c, const double *w, int nrep, double *ms_out, int nmax, void *stream) {
  if (!c || c->batch || c->kin || !w || !ms_out || nmax < 1 || nrep < 1) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  const bool f64 = c->prec == DG_FP64;
  const int nk = f64 ? 2 : 5;
  // FP32-bulk kind 4 writes an FP64 state: into a temporary, not the caller's w
  double *tmp64 = nullptr;
  if (!f64 && nmax > 4 && cudaMalloc(&tmp64, c->len * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  // Each kind runs nrep times back to back between two events (as in a step,
  // where the kernels follow each other in a graph): the mean includes the
  // gap between dependent launches but no per-launch event overhead.
  auto launch = [&](int k) {
    if (f64) {
      if (k == 0) c->ks.volume(c->prm, w, c->d_rvol, c->d_trace, s);
      else c->ks.surface(c->prm, MODE_RHS, 0.0, w, w, c->d_rvol, c->d_trace, c->d_w1, s);
    } else if (k == 0) {  // the kernels of a step as dg_step launches them (FP32 state in, FP32 stage out)
      c->ks32.volume(c->prm, c->pf, c->d_opsf, c->d_hi32[0], c->d_rvol32, c->d_trace32, nullptr, nullptr, nullptr,
                     nullptr, s);
    } else if (k == 1) {
      const StageIO io{c->d_hi32[0], nullptr, c->d_dd32[0], c->d_dd32[1], nullptr, nullptr, nullptr, nullptr};
      c->ks32.surface(c->prm, c->pf, c->d_opsf, MODE_S2, 1e-9f, io, c->d_rvol32, c->d_trace32, s);
    } else if (k == 2) {
      const StageIO io{c->d_hi32[0], nullptr, c->d_dd32[0], c->d_dd32[1], nullptr, nullptr, nullptr, nullptr};
      c->ks32.surfvol(c->prm, c->pf, c->d_opsf, MODE_S2, 1e-9f, io, c->d_rvol32, c->d_trace32, c->d_rvol32b,
                      c->d_trace32b, s);
    } else if (k == 3) {  // the first stage of a single-step call: reads the FP64 state (hi part only)
      c->ks32.volume(c->prm, c->pf, c->d_opsf, nullptr, c->d_rvol32b, c->d_trace32b, w, c->d_hi32[1], nullptr,
                     nullptr, s);
    } else {  // the last stage of a single-step call: adds the last increment to the FP64 state
      const StageIO io{nullptr, nullptr, c->d_dd32[0], nullptr, nullptr, nullptr, tmp64, w};
      c->ks32.surface(c->prm, c->pf, c->d_opsf, MODE_S3, 1e-9f, io, c->d_rvol32, c->d_trace32, s);
    }
  };
  if (!f64) {  // the internal state of w (hi, lo) and a zero increment to time the stage kernels on
    c->ks32.volume(c->prm, c->pf, c->d_opsf, nullptr, c->d_rvol32, c->d_trace32, w, c->d_hi32[0], c->d_lo32[0],
                   nullptr, s);
    cudaMemsetAsync(c->d_dd32[0], 0, (size_t)SW32 * c->N * sizeof(float), s);
  }
  cudaEvent_t ev[2];
  for (auto &x : ev) cudaEventCreate(&x);
  for (int k = 0; k < std::min(nk, nmax); ++k) {
    launch(k);  // warm-up
    cudaEventRecord(ev[0], s);
    for (int r = 0; r < nrep; ++r) launch(k);
    cudaEventRecord(ev[1], s);
    cudaEventSynchronize(ev[1]);
    float t = 0.f;
    cudaEventElapsedTime(&t, ev[0], ev[1]);
    if (k < nmax) ms_out[k] = (double)t / nrep;
  }
  for (auto &x : ev) cudaEventDestroy(x);
  cudaFree(tmp64);
  if (cudaGetLastError() != cudaSuccess) return -1;
  return std::min(nmax, nk);
}

extern "C" int dg_step_launches(const dg_ctx *c, int nsteps) {
  if (!c || c->batch || c->kin || nsteps < 0) return -1;
  if (nsteps == 0) return 0;
  return c->prec == DG_FP64 ? 6 * nsteps : 1 + 3 * nsteps;  // enqueue_step, enqueue_steps32
}

extern "C" int dg_kernel_costs(const dg_ctx *c, double *flops, double *bytes, int nmax) {
  if (!c || c->batch || c->kin || !flops || !bytes || nmax < 1) return -1;
  // Algorithmic counts from the formulas of the scheme (an FMA counts 2, a
  // division or square root 1), per launch.
  const double P1 = c->P1, Np = c->Np, NFK = c->NFK, E = c->E, d = c->dim;
  const double fface = NFK / Np;  // face nodes per node (upper bound of trace writers)
  const bool visc = c->opts.viscous != 0, st = c->opts.surface_tension != 0;
  // volume kernel, per node: closure 25, gradients 2*2*d*P1 (+4*d*P1 viscous),
  // normal 6, a_1 10, fluxes 40, volume contractions 2*6*d*P1, non-conservative 8,
  // sound speed at face nodes 5
  double fv = 25 + 4 * d * P1 + 6 + 10 + 40 + 12 * d * P1 + 8 + 5 * fface;
  if (visc) fv += 4 * d * P1 + 20 + 12;
  if (st) fv += 2 * d * P1 + 8;
  // surface kernel: per face node 133 (+30 viscous); per node gather/lift/update ~104
  double fs = fface * (133 + (visc ? 30 : 0)) + 7 * fface + 12 * 2 * d + 14 + 35;
  // Bytes: the volume kernel reads the state and writes the volume part and
  // the face traces; the surface kernel reads both traces of every face node,
  // the volume part, the stage input and the step start (FP32-bulk: the step
  // start and the previous increment), and writes the stage (FP32-bulk: its
  // increment).  FP32-bulk stores traces as padded 12-word records and, in the
  // inviscid kernels, the state and volume parts as padded 8-word node records.
  const bool f64 = c->prec == DG_FP64;
  const double nt = f64 ? c->ks.nt : TRW32;
  const double nw = f64 || visc ? 7 : SW32;
  const double word = f64 ? 8.0 : 4.0;
  if (!f64) fv += 3 * 2 * d * P1;  // compression term of the reduced energy
  const double bv = word * (E * Np * (nw + nw) + E * NFK * nt);
  const double bs = word * (E * NFK * nt * 2 + E * Np * (nw * 4));
  // The fused FP32-bulk stage kernel does both; its volume part takes the
  // stage state from registers instead of reading it back.
  const double bsv = bv + bs - word * E * Np * nw;
  // FP32-bulk kinds 3 and 4, a call's first volume kernel (reads the FP64 state, writes hi and lo,
  // 3 FP64 operations per variable for the split) and last surface kernel (reads the step start's
  // hi and lo, writes the FP64 state hi + lo: 9 operations of the float-float sum and 2 for the
  // sum per variable)
  const double b3 = 8.0 * NV * E * Np + 4.0 * (E * Np * 3 * nw + E * NFK * nt);
  const double b4 = 4.0 * (E * NFK * nt * 2 + E * Np * 4 * nw) + 8.0 * NV * E * Np;
  const int nk = std::min(nmax, c->prec == DG_FP64 ? 2 : 5);
  const double F[5] = {fv * E * Np, fs * E * Np, (fv + fs) * E * Np, (fv + 3 * NV) * E * Np, (fs + 11 * NV) * E * Np};
  const double Bb[5] = {bv, bs, bsv, b3, b4};
  for (int k = 0; k < nk; ++k) {
    flops[k] = F[k];
    bytes[k] = Bb[k];
  }
  return nk;
}

// ---------------------------------------------------------------------------
// Batched ensemble (FP32-bulk)
// ---------------------------------------------------------------------------

extern "C" dg_status dg_batch_create(int n, const dg_mesh *meshes, const int *p, const dg_eos *eos,
                                     const double *Gamma, const double *eps, const dg_opts *opts, dg_ctx **out) {
  if (!out) return fail(nullptr, DG_ERR_ARG, "dg_batch_create: out is NULL");
  *out = nullptr;
  if (n < 1 || !meshes || !p || !eos || !Gamma || !eps)
    return fail(nullptr, DG_ERR_ARG, "dg_batch_create: need n >= 1 and all arrays");
  const dg_opts o = normalised_opts(opts);
  if (o.prec != DG_FP32_BULK)
    return fail(nullptr, DG_ERR_UNSUPPORTED, "dg_batch_create: the batched form runs the FP32-bulk path only");
  if (o.viscous || o.surface_tension || o.grad_lift)
    return fail(nullptr, DG_ERR_UNSUPPORTED,
                "dg_batch_create: viscous and surface-tension terms and lifted gradients are not batched");
  if (o.batch_tile < 0 || o.batch_tile > NVAR)
    return fail(nullptr, DG_ERR_ARG, "dg_batch_create: batch_tile must be 0 (tune) or 1..4");
  for (int k = 0; k < n; ++k) {
    dg_status code;
    if (const char *why = check_problem(meshes + k, p[k], eos + k, Gamma[k], eps[k], &code))
      return fail(nullptr, code, "dg_batch_create: problem " + std::to_string(k) + ": " + why);
    if (meshes[k].dim != 2)
      return fail(nullptr, DG_ERR_UNSUPPORTED, "dg_batch_create: the batched form is two-dimensional");
  }
  dg_ctx *c = new (std::nothrow) dg_ctx();
  BatchData *b = c ? new (std::nothrow) BatchData() : nullptr;
  if (!c || !b) {
    delete c;
    return fail(nullptr, DG_ERR_OOM, "dg_batch_create: host allocation failed");
  }
  c->batch = b;
  c->opts = o;
  c->prec = DG_FP32_BULK;
  b->n = n;
  b->h.resize(n);
  b->group_of.assign(n, -1);
  b->slot_of.assign(n, -1);
  b->len.resize(n);

  // Groups by order, problems in the given order within a group.
  for (int k = 0; k < n; ++k) {
    int g = -1;
    for (size_t q = 0; q < b->groups.size(); ++q)
      if (b->groups[q].p == p[k]) g = (int)q;
    if (g < 0) {
      BatchGroup grp;
      grp.p = p[k];
      if (!batch_variants(p[k], grp.var)) {
        free_ctx(c);
        return fail(nullptr, DG_ERR_UNSUPPORTED, "dg_batch_create: order not available");
      }
      b->groups.push_back(grp);
      g = (int)b->groups.size() - 1;
    }
    b->group_of[k] = g;
    b->slot_of[k] = (int)b->groups[g].probs.size();
    b->groups[g].probs.push_back(k);
  }

  // One pool for every FP32 buffer and table: per problem the table, the
  // internal state, the two stage increments, the volume parts and the face
  // traces.
  std::vector<std::vector<float>> tables(n);
  std::vector<size_t> off(n);
  size_t total = 0;
  auto take = [&](size_t floats) {
    const size_t at = total;
    total += (floats + 63) & ~size_t(63);  // 256-byte aligned slices
    return at;
  };
  std::vector<size_t> o_ops(n), o_ws(n), o_d1(n), o_d2(n), o_rv(n), o_tr(n), o_rv2(n), o_tr2(n);
  for (int k = 0; k < n; ++k) {
    const dg_mesh &m = meshes[k];
    const double hx = (m.x1 - m.x0) / m.nx, hy = (m.y1 - m.y0) / m.ny;
    const std::vector<double> ops = build_ops(2, p[k], hx, hy);
    tables[k].assign(ops.begin(), ops.end());
    BatchProb &d = b->h[k];
    d.prm = make_params(&m, p[k], eos + k, Gamma[k], eps[k], o, hx, hy);
    d.prm.check_finite = 0;
    d.pf = to_float(d.prm);
    const size_t E = (size_t)m.nx * m.ny, P1 = p[k] + 1, NFK = 4 * P1;
    const size_t len = NV * E * P1 * P1, len32 = SW32 * E * P1 * P1;  // FP64 state; FP32 node records
    b->len[k] = len;
    o_ops[k] = take(tables[k].size());
    o_ws[k] = take(len32);
    o_d1[k] = take(len32);
    o_d2[k] = take(len32);
    o_rv[k] = take(len32);
    o_tr[k] = take((size_t)TRW32 * E * NFK);
    o_rv2[k] = take(len32);
    o_tr2[k] = take((size_t)TRW32 * E * NFK);
  }
  cudaError_t e = cudaMalloc(&b->d_pool, total * sizeof(float));
  if (e != cudaSuccess) {
    free_ctx(c);
    cudaGetLastError();
    return fail(nullptr, e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA,
                std::string("dg_batch_create: device allocation failed: ") + cudaGetErrorString(e));
  }
  float *pool = static_cast<float *>(b->d_pool);
  for (int k = 0; k < n && e == cudaSuccess; ++k) {
    BatchProb &d = b->h[k];
    d.opsf = pool + o_ops[k];
    d.ws = pool + o_ws[k];
    d.d1 = pool + o_d1[k];
    d.d2 = pool + o_d2[k];
    d.rvol[0] = pool + o_rv[k];
    d.tr[0] = pool + o_tr[k];
    d.rvol[1] = pool + o_rv2[k];
    d.tr[1] = pool + o_tr2[k];
    d.w64 = nullptr;
    d.dt = 0.f;
    d.prm.ops = nullptr;
    d.prm.status = nullptr;
    e = cudaMemcpy(pool + o_ops[k], tables[k].data(), tables[k].size() * sizeof(float), cudaMemcpyHostToDevice);
  }
  for (auto &g : b->groups) {
    if (e != cudaSuccess) break;
    if ((e = cudaMalloc(&g.d_probs, g.probs.size() * sizeof(BatchProb))) != cudaSuccess) break;
    for (int v = 0; v < NVAR && e == cudaSuccess; ++v) {
      std::vector<int> block0(g.probs.size());
      int nb = 0;
      for (size_t q = 0; q < g.probs.size(); ++q) {
        block0[q] = nb;
        nb += (b->h[g.probs[q]].prm.E + g.var[v].epb - 1) / g.var[v].epb;
      }
      g.nblocks[v] = nb;
      if ((e = cudaMalloc(&g.d_block0[v], g.probs.size() * sizeof(int))) != cudaSuccess) break;
      e = cudaMemcpy(g.d_block0[v], block0.data(), block0.size() * sizeof(int), cudaMemcpyHostToDevice);
    }
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  // the status word: the batched kernels latch no value checks (check_finite is off), only the
  // index checks of the bounds-checked build
  if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(unsigned));
  for (int k = 0; k < n && e == cudaSuccess; ++k) b->h[k].prm.status = c->d_status;
  for (auto &g : b->groups) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    free_ctx(c);
    cudaGetLastError();
    return fail(nullptr, DG_ERR_CUDA, std::string("dg_batch_create: ") + cudaGetErrorString(e));
  }
  c->len = 0;
  for (int k = 0; k < n; ++k) c->len += b->len[k];
  *out = c;
  return DG_OK;
}

// Upload the descriptors of every group (pageable source: the copy has read
// the host data when the call returns).
static dg_status upload_descriptors(dg_ctx *c, cudaStream_t s) {
  BatchData *b = c->batch;
  for (auto &g : b->groups) {
    std::vector<BatchProb> tmp(g.probs.size());
    for (size_t q = 0; q < g.probs.size(); ++q) tmp[q] = b->h[g.probs[q]];
    const cudaError_t e =
        cudaMemcpyAsync(g.d_probs, tmp.data(), tmp.size() * sizeof(BatchProb), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "dg_batch_step: descriptor upload");
  }
  return DG_OK;
}

// The first `nk` kernels of one step of one order group in tile variant v:
// volume part of stage 1, two fused stage kernels, surface part of stage 3.
static dg_status enqueue_group_step(dg_ctx *c, const BatchGroup &g, int v, cudaStream_t s, int nk = 4) {
  const int kind[4] = {BK_VOLUME, BK_SURFVOL, BK_SURFVOL, BK_SURFACE};
  for (int q = 0; q < nk; ++q) {
    cudaError_t e = g.var[v].launch(kind[q], g.d_probs, g.d_block0[v], (int)g.probs.size(), q, g.nblocks[v], s);
    if (e != cudaSuccess) return cuda_fail(c, e, "batched stage kernel launch");
  }
  return DG_OK;
}

// Tile autotuner: time every variant of every order group on the batch
// itself -- the stage-1 volume kernel and the two fused kernels, which read
// the caller's states and write only internal buffers -- and keep the
// fastest.  Runs once, before the first step's graphs are captured.
static dg_status tune_batch(dg_ctx *c, cudaStream_t s) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "dg_batch_step: tuning");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(c, cudaGetLastError(), "dg_batch_step: tuning");
  }
  dg_status r = DG_OK;
  const int reps = 3;
  if (c->opts.batch_tile > 0) {  // fixed by the caller: no timing
    for (auto &g : c->batch->groups) g.best = c->opts.batch_tile - 1;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return DG_OK;
  }
  for (auto &g : c->batch->groups) {
    for (int v = 0; v < NVAR && r == DG_OK; ++v) {
      r = enqueue_group_step(c, g, v, s, 3);  // warm-up
      cudaEventRecord(e0, s);
      for (int k = 0; k < reps && r == DG_OK; ++k) r = enqueue_group_step(c, g, v, s, 3);
      cudaEventRecord(e1, s);
      const cudaError_t e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        if (r == DG_OK) r = cuda_fail(c, e != cudaSuccess ? e : cudaGetLastError(), "dg_batch_step: tuning");
        break;
      }
      g.ms[v] = ms / reps;
    }
    if (r != DG_OK) break;
    g.best = 0;
    for (int v = 1; v < NVAR; ++v)
      if (g.ms[v] < g.ms[g.best]) g.best = v;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return r;
}

// The order groups share no data, so the captured graph holds one branch per
// group (forked from and joined back to the capture stream): the groups' kernels
// run concurrently and fill each other's tails.
static dg_status capture_batch(dg_ctx *c, int steps, cudaGraphExec_t *exec) {
  BatchData *b = c->batch;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_batch_step: begin capture");
  dg_status r = DG_OK;
  e = cudaEventRecord(b->fork, c->cap);
  for (auto &grp : b->groups) {
    if (e == cudaSuccess) e = cudaStreamWaitEvent(grp.stream, b->fork, 0);
    for (int k = 0; k < steps && e == cudaSuccess && r == DG_OK; ++k)
      r = enqueue_group_step(c, grp, grp.best, grp.stream);
    if (e == cudaSuccess) e = cudaEventRecord(grp.done, grp.stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->cap, grp.done, 0);
  }
  const cudaError_t e_end = cudaStreamEndCapture(c->cap, &g);
  if (r != DG_OK || e != cudaSuccess || e_end != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (r != DG_OK) return r;
    return cuda_fail(c, e != cudaSuccess ? e : e_end, "dg_batch_step: capture");
  }
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  return e == cudaSuccess ? DG_OK : cuda_fail(c, e, "dg_batch_step: instantiate");
}

extern "C" int dg_batch_tiles(const dg_ctx *c, int *p, int *epb, int *minb, double *ms_best, double *ms_default,
                              int nmax) {
  if (!c || !c->batch || nmax < 0) return -1;
  int n = 0;
  for (const auto &g : c->batch->groups) {
    if (g.best < 0) return 0;
    if (n < nmax) {
      if (p) p[n] = g.p;
      if (epb) epb[n] = g.var[g.best].epb;
      if (minb) minb[n] = g.var[g.best].minb;
      if (ms_best) ms_best[n] = g.ms[g.best];
      if (ms_default) ms_default[n] = g.ms[0];
    }
    ++n;
  }
  return std::min(n, nmax);
}

extern "C" dg_status dg_batch_step(dg_ctx *c, double *const *w, const double *dt, int nsteps, void *stream) {
  if (!c) return DG_ERR_ARG;
  if (!c->batch) return fail(c, DG_ERR_ARG, "dg_batch_step: context was not made by dg_batch_create");
  if (!w || !dt || nsteps < 0) return fail(c, DG_ERR_ARG, "dg_batch_step: need w, dt and nsteps >= 0");
  BatchData *b = c->batch;
  bool changed = false;
  for (int k = 0; k < b->n; ++k) {
    if (!w[k] || !(dt[k] > 0.0)) return fail(c, DG_ERR_ARG, "dg_batch_step: null state or dt <= 0");
    if (b->h[k].w64 != w[k] || b->h[k].dt != (float)dt[k]) changed = true;
    b->h[k].w64 = w[k];
    b->h[k].dt = (float)dt[k];
  }
  if (nsteps == 0) return DG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (changed) {
    const dg_status r = upload_descriptors(c, s);
    if (r != DG_OK) return r;
  }
  if (!c->g1) {  // the graphs read the descriptors at run time: captured once
    dg_status r;
    if ((r = tune_batch(c, s)) != DG_OK) return r;
    if ((r = capture_batch(c, 1, &c->g1)) != DG_OK) return r;
    if ((r = capture_batch(c, GRAPH_UNROLL, &c->gk)) != DG_OK) return r;
  }
  cudaError_t e;
  for (int k = 0; k < nsteps / GRAPH_UNROLL; ++k)
    if ((e = cudaGraphLaunch(c->gk, s)) != cudaSuccess) return cuda_fail(c, e, "dg_batch_step: graph launch");
  for (int k = 0; k < nsteps % GRAPH_UNROLL; ++k)
    if ((e = cudaGraphLaunch(c->g1, s)) != cudaSuccess) return cuda_fail(c, e, "dg_batch_step: graph launch");
  return DG_OK;
}

// ---------------------------------------------------------------------------
// Kinematic mode (Sec. 4.1)
// ---------------------------------------------------------------------------

namespace dgpf {
__global__ void k_kin_set_time(double *t0, double t);
}

extern "C" dg_status dg_kin_create(const dg_mesh *mesh, int p, double Gamma, double eps, const dg_velocity *vel,
                                   double c_ip, dg_ctx **out) {
  if (!out) return fail(nullptr, DG_ERR_ARG, "dg_kin_create: out is NULL");
  *out = nullptr;
  if (!mesh || !vel) return fail(nullptr, DG_ERR_ARG, "dg_kin_create: mesh and velocity are required");
  if (mesh->dim != 2) return fail(nullptr, DG_ERR_ARG, "dg_kin_create: the kinematic mode is two-dimensional");
  if (mesh->elem != DG_ELEM_QUAD && mesh->elem != DG_ELEM_TRI)
    return fail(nullptr, DG_ERR_ARG, "dg_kin_create: elem must be DG_ELEM_QUAD or DG_ELEM_TRI");
  const bool tri = mesh->elem == DG_ELEM_TRI;
  if (p < 1 || p > (tri ? 4 : 5))
    return fail(nullptr, DG_ERR_UNSUPPORTED,
                tri ? "dg_kin_create: order p must be in 1..4 on triangles" : "dg_kin_create: order p must be in 1..5");
  if (mesh->nx < 1 || mesh->ny < 1 || (long long)mesh->nx * mesh->ny > (1LL << 26))
    return fail(nullptr, DG_ERR_ARG, "dg_kin_create: need 1 <= nx, ny and a mesh of at most 2^26 elements");
  // nodes per field must fit the kernels' 32-bit node count
  const long long nodes = (long long)mesh->nx * mesh->ny * (tri ? 2LL * (p + 1) * (p + 2) / 2 : (p + 1LL) * (p + 1));
  if (nodes >= (1LL << 31))
    return fail(nullptr, DG_ERR_ARG, "dg_kin_create: problem too large for one context (2^31 nodes per field)");
  if (!(mesh->x1 > mesh->x0) || !(mesh->y1 > mesh->y0)) return fail(nullptr, DG_ERR_ARG, "dg_kin_create: empty domain");
  for (int f = 0; f < 4; ++f)
    if (mesh->bc[f] != DG_BC_PERIODIC)
      return fail(nullptr, DG_ERR_UNSUPPORTED, "dg_kin_create: periodic boundaries only");
  if (!(Gamma >= 0.0) || !(eps >= 0.0)) return fail(nullptr, DG_ERR_ARG, "dg_kin_create: need Gamma, eps >= 0");
  if (vel->kind != DG_VEL_UNIFORM && vel->kind != DG_VEL_RIDER_KOTHE)
    return fail(nullptr, DG_ERR_ARG, "dg_kin_create: unknown velocity kind");
  if (vel->kind == DG_VEL_RIDER_KOTHE && !(vel->T > 0.0))
    return fail(nullptr, DG_ERR_ARG, "dg_kin_create: the Rider-Kothe period must be > 0");
  dg_ctx *c = new (std::nothrow) dg_ctx();
  if (!c) return fail(nullptr, DG_ERR_OOM, "dg_kin_create: host allocation failed");
  c->kin = true;
  c->tri = tri;
  c->mesh = *mesh;
  c->p = p;
  c->dim = 2;
  c->P1 = p + 1;
  c->Np = tri ? (p + 1) * (p + 2) / 2 : c->P1 * c->P1;
  c->E = (tri ? 2 : 1) * mesh->nx * mesh->ny;
  c->N = c->E * c->Np;
  c->NFK = tri ? 3 * (p + 2) : 4 * c->P1;
  c->len = (size_t)2 * c->N;
  c->hx = (mesh->x1 - mesh->x0) / mesh->nx;
  c->hy = (mesh->y1 - mesh->y0) / mesh->ny;
  if (tri ? !tri_kernels(p, &c->tk) : !kin_kernels(p, &c->kk)) {
    free_ctx(c);
    return fail(nullptr, DG_ERR_UNSUPPORTED, "dg_kin_create: order not available");
  }
  const double cip = c_ip > 0.0 ? c_ip : 1.0;
  KinParams &k = c->kp;
  k.nx = mesh->nx;
  k.ny = mesh->ny;
  k.E = c->E;
  k.N = c->N;
  k.x0 = mesh->x0;
  k.y0 = mesh->y0;
  k.hx = c->hx;
  k.hy = c->hy;
  k.Gamma = Gamma;
  k.eps = eps;
  k.eta_x = cip * c->P1 * c->P1 / c->hx;
  k.eta_y = cip * c->P1 * c->P1 / c->hy;
  k.eta_tri = cip * (p + 1) * (p + 2);
  if (tri) tri_constants(c->hx, c->hy, k.eta_tri, k.tc);
  k.vel = vel->kind;
  k.u0 = vel->u0;
  k.v0 = vel->v0;
  k.T = vel->T;
  k.xc = vel->xc;
  k.yc = vel->yc;
  k.check_finite = 1;
  const std::vector<double> ops = tri ? tri_tables(p, k.tc) : build_ops(2, p, c->hx, c->hy);
  if (ops.empty()) {
    free_ctx(c);
    return fail(nullptr, DG_ERR_UNSUPPORTED, "dg_kin_create: reference tables could not be built");
  }
  std::vector<double> xi, wt;
  gll_nodes(p, xi, wt);
  const size_t sb = c->len * sizeof(double);
  cudaError_t e = cudaSuccess;
  // one kernel per stage on either element type: no volume residual or face traces in memory
  double **bufs[] = {&c->d_kacc, &c->d_kwsA, &c->d_kwsB};
  for (double **b : bufs)
    if (e == cudaSuccess) e = cudaMalloc(b, sb);
  // the velocity's spatial factor at every node (rectangles) or quadrature point (triangles)
  const size_t vrows = tri ? (size_t)c->E * c->tk.points : (size_t)c->N;
  if (e == cudaSuccess) e = cudaMalloc(&c->d_ktv, 2 * vrows * sizeof(double));
  if (e == cudaSuccess && tri) {
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c->tk.fn, c->tk.threads, 0);
    const long groups = (c->E + tri_group(p) - 1) / tri_group(p);
    c->tri_grid = (int)std::max(1L, std::min(groups, (long)std::max(1, sms) * std::max(1, per_sm)));
  }
  if (e == cudaSuccess) e = cudaMalloc(&c->d_kt0, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_dt, sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(c->d_dt, 0, sizeof(double));  // dg_kin_rhs: stage time t0 exactly
  if (e == cudaSuccess) e = cudaMalloc(&c->d_kxi, xi.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_ops, ops.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemcpy(c->d_ops, ops.data(), ops.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_kxi, xi.data(), xi.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c->d_kt0, 0, sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    free_ctx(c);
    cudaGetLastError();
    return fail(nullptr, e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA,
                std::string("dg_kin_create: ") + cudaGetErrorString(e));
  }
  k.ops = c->d_ops;
  k.xi = c->d_kxi;
  k.t0 = c->d_kt0;
  k.dt = c->d_dt;
  k.status = c->d_status;
  k.vel_tab = c->d_ktv;
  e = tri ? c->tk.velocity_table(k, c->d_ktv, c->cap) : c->kk.velocity_table(k, c->d_ktv, c->cap);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->cap);
  if (e != cudaSuccess) {
    free_ctx(c);
    cudaGetLastError();
    return fail(nullptr, DG_ERR_CUDA, std::string("dg_kin_create: velocity table: ") + cudaGetErrorString(e));
  }
  *out = c;
  return DG_OK;
}

static dg_status kin_check(dg_ctx *c, const char *who) {
  if (!c) return DG_ERR_ARG;
  if (!c->kin) return fail(c, DG_ERR_ARG, std::string(who) + ": not a kinematic context (dg_kin_create)");
  return DG_OK;
}

extern "C" dg_status dg_kin_nodes(const dg_mesh *mesh, int p, double *x, double *y) {
  if (!mesh || !x || !y) return fail(nullptr, DG_ERR_ARG, "dg_kin_nodes: mesh, x and y are required");
  if (mesh->dim != 2 || mesh->nx < 1 || mesh->ny < 1 || !(mesh->x1 > mesh->x0) || !(mesh->y1 > mesh->y0))
    return fail(nullptr, DG_ERR_ARG, "dg_kin_nodes: need a non-empty 2D mesh");
  if (mesh->elem != DG_ELEM_QUAD && mesh->elem != DG_ELEM_TRI)
    return fail(nullptr, DG_ERR_ARG, "dg_kin_nodes: elem must be DG_ELEM_QUAD or DG_ELEM_TRI");
  const bool tri = mesh->elem == DG_ELEM_TRI;
  if (p < 1 || p > (tri ? 4 : 5)) return fail(nullptr, DG_ERR_UNSUPPORTED, "dg_kin_nodes: order out of range");
  const double hx = (mesh->x1 - mesh->x0) / mesh->nx, hy = (mesh->y1 - mesh->y0) / mesh->ny;
  long n = 0;
  if (!tri) {
    std::vector<double> xi, wt;
    gll_nodes(p, xi, wt);
    for (int ey = 0; ey < mesh->ny; ++ey)
      for (int ex = 0; ex < mesh->nx; ++ex)
        for (int j = 0; j <= p; ++j)
          for (int i = 0; i <= p; ++i, ++n) {
            x[n] = mesh->x0 + hx * (ex + 0.5 * (xi[i] + 1.0));
            y[n] = mesh->y0 + hy * (ey + 0.5 * (xi[j] + 1.0));
          }
    return DG_OK;
  }
  for (int cell = 0; cell < mesh->nx * mesh->ny; ++cell)
    for (int type = 0; type < 2; ++type) {
      const double xa = mesh->x0 + (cell % mesh->nx) * hx, ya = mesh->y0 + (cell / mesh->nx) * hy;
      const double v[3][2] = {{xa, ya},
                              {xa + hx, type == 0 ? ya : ya + hy},
                              {type == 0 ? xa + hx : xa, ya + hy}};
      for (int j = 0; j <= p; ++j)
        for (int i = 0; i + j <= p; ++i, ++n) {
          const double r = -1.0 + 2.0 * i / p, s = -1.0 + 2.0 * j / p;
          x[n] = v[0][0] + 0.5 * (1.0 + r) * (v[1][0] - v[0][0]) + 0.5 * (1.0 + s) * (v[2][0] - v[0][0]);
          y[n] = v[0][1] + 0.5 * (1.0 + r) * (v[1][1] - v[0][1]) + 0.5 * (1.0 + s) * (v[2][1] - v[0][1]);
        }
    }
  return DG_OK;
}

extern "C" dg_status dg_kin_rhs(dg_ctx *c, const double *w, double t, double *L, void *stream) {
  dg_status r = kin_check(c, "dg_kin_rhs");
  if (r != DG_OK) return r;
  if (!w || !L || w == L) return fail(c, DG_ERR_ARG, "dg_kin_rhs: need distinct, non-null w and L");
  cudaStream_t s = (cudaStream_t)stream;
  k_kin_set_time<<<1, 1, 0, s>>>(c->d_kt0, t);
  cudaError_t e = cudaGetLastError();
  if (c->tri) {
    if (e == cudaSuccess) e = c->tk.stage(c->kp, KIN_RHS, 0, 0.0, w, nullptr, nullptr, L, c->tri_grid, s);
    return e == cudaSuccess ? DG_OK : cuda_fail(c, e, "dg_kin_rhs: launch");
  }
  if (e == cudaSuccess) e = c->kk.stage(c->kp, KIN_RHS, 0, 0.0, w, nullptr, nullptr, L, s);
  return e == cudaSuccess ? DG_OK : cuda_fail(c, e, "dg_kin_rhs: launch");
}

// One classical RK4 step of the captured sequence: step k of the graph, stage
// inputs w -> A -> B -> A, the last stage writes w in place.  The kernels read
// the step size from device memory (c->d_dt) and form the stage times there.
static dg_status enqueue_kin_step(dg_ctx *c, double *w, int k, cudaStream_t s) {
  double *A = c->d_kwsA, *B = c->d_kwsB;
  const double frac[4] = {0.0, 0.5, 0.5, 1.0};
  const double *in[4] = {w, A, B, A};
  double *out[4] = {A, B, A, w};
  const int mode[4] = {KIN_K1, KIN_K2, KIN_K3, KIN_K4};
  for (int st = 0; st < 4; ++st) {
    cudaError_t e;
    if (c->tri) {
      e = c->tk.stage(c->kp, mode[st], k, frac[st], in[st], w, c->d_kacc, out[st], c->tri_grid, s);
    } else {
      e = c->kk.stage(c->kp, mode[st], k, frac[st], in[st], w, c->d_kacc, out[st], s);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "dg_kin_step: launch");
  }
  return DG_OK;
}

static dg_status capture_kin(dg_ctx *c, double *w, int steps, cudaGraphExec_t *exec) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_kin_step: begin capture");
  dg_status r = DG_OK;
  for (int k = 0; k < steps && r == DG_OK; ++k) r = enqueue_kin_step(c, w, k, c->cap);
  e = cudaStreamEndCapture(c->cap, &g);
  if (r != DG_OK) {
    if (g) cudaGraphDestroy(g);
    return r;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_kin_step: end capture");
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  return e == cudaSuccess ? DG_OK : cuda_fail(c, e, "dg_kin_step: instantiate");
}

extern "C" dg_status dg_kin_step(dg_ctx *c, double *w, double t0, double dt, int nsteps, void *stream) {
  dg_status r = kin_check(c, "dg_kin_step");
  if (r != DG_OK) return r;
  if (!w) return fail(c, DG_ERR_ARG, "dg_kin_step: null state");
  if (!(dt > 0.0) || nsteps < 0) return fail(c, DG_ERR_ARG, "dg_kin_step: need dt > 0 and nsteps >= 0");
  if (nsteps == 0) return DG_OK;
  if (c->g_w != w || !c->g1) {  // the graphs read dt and the start time from device memory
    free_graphs(c);
    if ((r = capture_kin(c, w, 1, &c->g1)) != DG_OK) return r;
    if ((r = capture_kin(c, w, GRAPH_UNROLL, &c->gk)) != DG_OK) return r;
    c->g_w = w;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (dt != c->dt_set) {
    k_set_double<<<1, 1, 0, s>>>(c->d_dt, dt);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "dg_kin_step: set dt");
    c->dt_set = dt;
  }
  int done = 0;
  while (done < nsteps && e == cudaSuccess) {
    const bool big = nsteps - done >= GRAPH_UNROLL;
    k_kin_set_time<<<1, 1, 0, s>>>(c->d_kt0, t0 + done * dt);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaGraphLaunch(big ? c->gk : c->g1, s);
    done += big ? GRAPH_UNROLL : 1;
  }
  return e == cudaSuccess ? DG_OK : cuda_fail(c, e, "dg_kin_step: launch");
}

// ---------------------------------------------------------------------------
// Level-set re-initialisation (end of Sec. 3)
// ---------------------------------------------------------------------------

extern "C" dg_status dg_reinit(dg_ctx *c, double *w, int niter, double nu, double dtau, void *stream) {
  if (!c) return DG_ERR_ARG;
  if (c->batch) return fail(c, DG_ERR_ARG, "dg_reinit: batch context");
  if (!w) return fail(c, DG_ERR_ARG, "dg_reinit: null state");
  if (niter < 0) return fail(c, DG_ERR_ARG, "dg_reinit: need niter >= 0");
  if (c->tri) return fail(c, DG_ERR_UNSUPPORTED, "dg_reinit: rectangular elements only");
  ReinitKernels rk;
  if (!reinit_kernels(c->p, c->dim, &rk)) return fail(c, DG_ERR_UNSUPPORTED, "dg_reinit: order not available");
  ReinitParams rp{};
  if (c->kin) {
    rp.nx = c->kp.nx;
    rp.ny = c->kp.ny;
    rp.E = c->kp.E;
    rp.N = c->kp.N;
    for (int f = 0; f < 4; ++f) rp.bc[f] = BC_PERIODIC;
    rp.eps = c->kp.eps;
    rp.eta_x = c->kp.eta_x;
    rp.eta_y = c->kp.eta_y;
  } else {
    rp.nx = c->prm.nx;
    rp.ny = c->prm.ny;
    rp.E = c->prm.E;
    rp.N = c->prm.N;
    for (int f = 0; f < 4; ++f) rp.bc[f] = c->prm.bc[f];
    rp.eps = c->prm.eps;
    rp.eta_x = c->prm.eta_x;
    rp.eta_y = c->prm.eta_y;
  }
  rp.ops = c->d_ops;
  rp.status = c->d_status;
  const double h = c->dim == 2 ? std::min(c->hx, c->hy) : c->hx;
  const double q = 2.0 * c->p + 1.0;
  rp.nu = nu > 0.0 ? nu : h / (2.0 * (c->p + 1));
  if (!(dtau > 0.0)) dtau = std::min(0.5 * h / q, 0.1 * h * h / (q * q * rp.nu));
  cudaError_t e = cudaSuccess;
  if (!c->d_riS) {
    const size_t nb = (size_t)rp.N * sizeof(double), tb = (size_t)2 * rp.E * rk.nfk * sizeof(double);
    double **bufs[] = {&c->d_riS, &c->d_ri1, &c->d_ri2, &c->d_rirvol};
    for (double **b : bufs)
      if (e == cudaSuccess) e = cudaMalloc(b, nb);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_ritr, tb);
    if (e != cudaSuccess) {
      for (double **b : {&c->d_riS, &c->d_ri1, &c->d_ri2, &c->d_rirvol, &c->d_ritr}) {
        cudaFree(*b);
        *b = nullptr;
      }
      cudaGetLastError();
      return fail(c, e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA,
                  std::string("dg_reinit: workspace: ") + cudaGetErrorString(e));
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  double *psi = w + rp.N;
  e = rk.sign(rp, w, c->d_riS, s);
  const int mode[3] = {MODE_S1, MODE_S2, MODE_S3};
  const double *in[3] = {psi, c->d_ri1, c->d_ri2};
  double *out[3] = {c->d_ri1, c->d_ri2, psi};
  for (int it = 0; it < niter && e == cudaSuccess; ++it)
    for (int st = 0; st < 3 && e == cudaSuccess; ++st) {
      e = rk.volume(rp, in[st], c->d_riS, c->d_rirvol, c->d_ritr, s);
      if (e == cudaSuccess) e = rk.surface(rp, mode[st], dtau, psi, in[st], c->d_rirvol, c->d_ritr, out[st], s);
    }
  return e == cudaSuccess ? DG_OK : cuda_fail(c, e, "dg_reinit: launch");
}

// ---------------------------------------------------------------------------
// Discrete adjoint (FP64, inviscid, no surface tension)
// ---------------------------------------------------------------------------

// out = ca xa + cb (dL/dw(w))^T lam + cc yc + cd zd
static dg_status run_vjp(dg_ctx *c, const double *w, const double *lam, double *out, double ca, const double *xa,
                         double cb, double cc, const double *yc, double cd, const double *zd, cudaStream_t s) {
  cudaError_t e = c->ks.volume(c->prm, w, c->d_rvol, c->d_trace, s);  // traces of w
  if (e == cudaSuccess) e = c->adj.face(c->prm, lam, c->d_trace, c->d_trbar, s);
  if (e == cudaSuccess) e = c->adj.volume(c->prm, w, lam, c->d_trbar, out, ca, xa, cb, cc, yc, cd, zd, s);
  return e == cudaSuccess ? DG_OK : cuda_fail(c, e, "adjoint kernel launch");
}

static dg_status adj_check(dg_ctx *c, const char *who) {
  if (c->batch) return fail(c, DG_ERR_ARG, std::string(who) + ": batch context");
  if (!c->has_adj)
    return fail(c, DG_ERR_UNSUPPORTED,
                std::string(who) + ": the adjoint covers the FP64 path without viscous and surface-tension terms");
  return DG_OK;
}

extern "C" dg_status dg_rhs_vjp(dg_ctx *c, const double *w, const double *lam, double *out, void *stream) {
  if (!c) return DG_ERR_ARG;
  dg_status r = adj_check(c, "dg_rhs_vjp");
  if (r != DG_OK) return r;
  if (!w || !lam || !out) return fail(c, DG_ERR_ARG, "dg_rhs_vjp: null array");
  if (out == w || out == lam) return fail(c, DG_ERR_ARG, "dg_rhs_vjp: out must not overlap w or lam");
  return run_vjp(c, w, lam, out, 0.0, nullptr, 1.0, 0.0, nullptr, 0.0, nullptr, (cudaStream_t)stream);
}

// Reverse of one SSP-RK3 step w_{n+1} = Phi(w_n) (Shu-Osher form):
//   w1 = w + dt L(w), w2 = 3/4 w + 1/4 (w1 + dt L(w1)), w3 = 1/3 w + 2/3 (w2 + dt L(w2)).
// Given lam3 = lam_{n+1}:
//   lam2 = 2/3 lam3 + 2/3 dt L'(w2)^T lam3
//   lam1 = 1/4 lam2 + 1/4 dt L'(w1)^T lam2
//   lam_n = lam1 + dt L'(w)^T lam1 + 1/3 lam3 + 3/4 lam2
// The stages w1, w2 are recomputed from w_n first.
extern "C" dg_status dg_adjoint_step(dg_ctx *c, const double *w_n, const double *lam_np1, double *lam_n, double dt,
                                     void *stream) {
  if (!c) return DG_ERR_ARG;
  dg_status r = adj_check(c, "dg_adjoint_step");
  if (r != DG_OK) return r;
  if (!w_n || !lam_np1 || !lam_n) return fail(c, DG_ERR_ARG, "dg_adjoint_step: null array");
  if (lam_n == w_n) return fail(c, DG_ERR_ARG, "dg_adjoint_step: lam_n must not overlap w_n");
  if (!(dt > 0.0)) return fail(c, DG_ERR_ARG, "dg_adjoint_step: need dt > 0");
  cudaStream_t s = (cudaStream_t)stream;
  if ((r = run_stage(c, MODE_S1, dt, w_n, w_n, c->d_w1, s)) != DG_OK) return r;
  if ((r = run_stage(c, MODE_S2, dt, w_n, c->d_w1, c->d_w2, s)) != DG_OK) return r;
  if ((r = run_vjp(c, c->d_w2, lam_np1, c->d_lam2, 2.0 / 3.0, lam_np1, 2.0 / 3.0 * dt, 0.0, nullptr, 0.0, nullptr,
                   s)) != DG_OK)
    return r;
  if ((r = run_vjp(c, c->d_w1, c->d_lam2, c->d_lam1, 0.25, c->d_lam2, 0.25 * dt, 0.0, nullptr, 0.0, nullptr, s)) !=
      DG_OK)
    return r;
  return run_vjp(c, w_n, c->d_lam1, lam_n, 1.0, c->d_lam1, dt, 1.0 / 3.0, lam_np1, 0.75, c->d_lam2, s);
}

// ---------------------------------------------------------------------------
// Taped step and its reverse (no recomputation in the reverse sweep)
// ---------------------------------------------------------------------------
// tape layout (doubles): w1 [7N] | w2 [7N] | traces of w, w1, w2 [3 x nt E NFK]

extern "C" size_t dg_tape_len(const dg_ctx *c) {
  if (!c || c->batch || !c->has_adj) return 0;
  return 2 * c->len + 3 * (size_t)c->ks.nt * c->E * c->NFK;
}

static void tape_parts(dg_ctx *c, double *tape, double **w1, double **w2, double **tr) {
  *w1 = tape;
  *w2 = tape + c->len;
  const size_t nt = (size_t)c->ks.nt * c->E * c->NFK;
  for (int k = 0; k < 3; ++k) tr[k] = tape + 2 * c->len + k * nt;
}

extern "C" dg_status dg_step_tape(dg_ctx *c, double *w, double dt, double *tape, void *stream) {
  if (!c) return DG_ERR_ARG;
  dg_status r = adj_check(c, "dg_step_tape");
  if (r != DG_OK) return r;
  if (!w || !tape) return fail(c, DG_ERR_ARG, "dg_step_tape: null array");
  if (!(dt > 0.0)) return fail(c, DG_ERR_ARG, "dg_step_tape: need dt > 0");
  cudaStream_t s = (cudaStream_t)stream;
  double *w1, *w2, *tr[3];
  tape_parts(c, tape, &w1, &w2, tr);
  const double *in[3] = {w, w1, w2};
  double *out[3] = {w1, w2, w};
  const int mode[3] = {MODE_S1, MODE_S2, MODE_S3};
  for (int k = 0; k < 3; ++k) {
    cudaError_t e = c->ks.volume(c->prm, in[k], c->d_rvol, tr[k], s);
    if (e == cudaSuccess) e = c->ks.surface(c->prm, mode[k], dt, w, in[k], c->d_rvol, tr[k], out[k], s);
    if (e != cudaSuccess) return cuda_fail(c, e, "dg_step_tape: kernel launch");
  }
  return DG_OK;
}

extern "C" dg_status dg_adjoint_step_tape(dg_ctx *c, const double *w_n, const double *tape, const double *lam_np1,
                                          double *lam_n, double dt, void *stream) {
  if (!c) return DG_ERR_ARG;
  dg_status r = adj_check(c, "dg_adjoint_step_tape");
  if (r != DG_OK) return r;
  if (!w_n || !tape || !lam_np1 || !lam_n) return fail(c, DG_ERR_ARG, "dg_adjoint_step_tape: null array");
  if (!(dt > 0.0)) return fail(c, DG_ERR_ARG, "dg_adjoint_step_tape: need dt > 0");
  cudaStream_t s = (cudaStream_t)stream;
  double *w1, *w2, *tr[3];
  tape_parts(c, const_cast<double *>(tape), &w1, &w2, tr);
  auto vjp = [&](const double *w, const double *trace, const double *lam, double *out, double ca, const double *xa,
                 double cb, double cc, const double *yc, double cd, const double *zd) {
    cudaError_t e = c->adj.face(c->prm, lam, trace, c->d_trbar, s);
    if (e == cudaSuccess) e = c->adj.volume(c->prm, w, lam, c->d_trbar, out, ca, xa, cb, cc, yc, cd, zd, s);
    return e;
  };
  cudaError_t e = vjp(w2, tr[2], lam_np1, c->d_lam2, 2.0 / 3.0, lam_np1, 2.0 / 3.0 * dt, 0.0, nullptr, 0.0, nullptr);
  if (e == cudaSuccess) e = vjp(w1, tr[1], c->d_lam2, c->d_lam1, 0.25, c->d_lam2, 0.25 * dt, 0.0, nullptr, 0.0, nullptr);
  if (e == cudaSuccess) e = vjp(w_n, tr[0], c->d_lam1, lam_n, 1.0, c->d_lam1, dt, 1.0 / 3.0, lam_np1, 0.75, c->d_lam2);
  return e == cudaSuccess ? DG_OK : cuda_fail(c, e, "dg_adjoint_step_tape: kernel launch");
}

// One checkpoint segment of a reverse sweep: replay m taped steps from
// states[0] (each step's start kept in states[j]), then m adjoint steps back
// through them, lam updated in place.  The whole sequence is one CUDA graph,
// captured on the first call for (m, dt, states, tapes, lam) and replayed.
static dg_status enqueue_segment(dg_ctx *c, int m, double dt, double *states, double *tapes, double *lam,
                                 cudaStream_t s) {
  const size_t len = c->len, tl = dg_tape_len(c);
  for (int j = 0; j < m; ++j) {
    cudaError_t e = cudaMemcpyAsync(states + (j + 1) * len, states + j * len, len * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "dg_adjoint_segment: copy");
    const dg_status r = dg_step_tape(c, states + (j + 1) * len, dt, tapes + j * tl, s);
    if (r != DG_OK) return r;
  }
  for (int j = m - 1; j >= 0; --j) {
    const dg_status r = dg_adjoint_step_tape(c, states + j * len, tapes + j * tl, lam, lam, dt, s);
    if (r != DG_OK) return r;
  }
  return DG_OK;
}

extern "C" dg_status dg_adjoint_segment(dg_ctx *c, const double *w_start, int m, double dt, double *states,
                                        double *tapes, double *lam, void *stream) {
  if (!c) return DG_ERR_ARG;
  dg_status r = adj_check(c, "dg_adjoint_segment");
  if (r != DG_OK) return r;
  if (!w_start || !states || !tapes || !lam) return fail(c, DG_ERR_ARG, "dg_adjoint_segment: null array");
  if (m < 1 || !(dt > 0.0)) return fail(c, DG_ERR_ARG, "dg_adjoint_segment: need m >= 1 and dt > 0");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(states, w_start, c->len * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_adjoint_segment: copy");
  dg_ctx::SegGraph *g = nullptr;
  for (auto &x : c->seg)
    if (x.exec && x.m == m && x.dt == dt && x.states == states && x.tapes == tapes && x.lam == lam) g = &x;
  if (!g) {
    g = !c->seg[0].exec ? &c->seg[0] : !c->seg[1].exec ? &c->seg[1] : &c->seg[0];
    if (g->exec) cudaGraphExecDestroy(g->exec);
    *g = dg_ctx::SegGraph{};
    cudaGraph_t graph = nullptr;
    if ((e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return cuda_fail(c, e, "dg_adjoint_segment: begin capture");
    r = enqueue_segment(c, m, dt, states, tapes, lam, c->cap);
    e = cudaStreamEndCapture(c->cap, &graph);
    if (r != DG_OK) {
      if (graph) cudaGraphDestroy(graph);
      return r;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "dg_adjoint_segment: end capture");
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g->exec = nullptr;
      return cuda_fail(c, e, "dg_adjoint_segment: instantiate");
    }
    g->m = m;
    g->dt = dt;
    g->states = states;
    g->tapes = tapes;
    g->lam = lam;
  }
  if ((e = cudaGraphLaunch(g->exec, s)) != cudaSuccess) return cuda_fail(c, e, "dg_adjoint_segment: graph launch");
  return DG_OK;
}
