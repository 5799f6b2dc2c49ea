// dg_noalloc.cu -- dg_rhs_noalloc: the FP64 right-hand side without any device
// allocation.
//
// For callers that must not call cudaMalloc (for example code running inside a
// framework's memory pool or under an allocator that forbids raw device
// allocations after start-up, or a process that has already reserved every
// byte of device memory): the caller passes only the state and the output; the
// operator table and the scratch the two kernels need (the volume part of
// M^-1 R and the face traces) live in one file-scope __device__ array of
// DG_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds until
// the process exits.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so the device address is looked up once per
// device with cudaGetSymbolAddress, with that device current, and cached.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "dg_common.cuh"
#include "dgpf.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[DG_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_addr[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// GLL nodes (Newton on (1 - x^2) P_p') and weights, into fixed-size arrays.
void gll(int p, double *x, double *w) {
  for (int i = 0; i <= p; ++i) x[i] = -std::cos(M_PI * i / p);
  for (int it = 0; it < 200; ++it) {
    double moved = 0.0;
    for (int i = 1; i < p; ++i) {
      double a = 1.0, b = x[i];
      for (int k = 2; k <= p; ++k) {
        const double c = ((2.0 * k - 1.0) * x[i] * b - (k - 1.0) * a) / k;
        a = b;
        b = c;
      }
      const double dx = (x[i] * b - a) / ((p + 1.0) * b);
      x[i] -= dx;
      moved = std::fmax(moved, std::fabs(dx));
    }
    if (moved < 1e-16) break;
  }
  for (int i = 0; i <= p / 2; ++i) {
    const double s = 0.5 * (x[p - i] - x[i]);
    x[i] = -s;
    x[p - i] = s;
  }
  if (p % 2 == 0) x[p / 2] = 0.0;
  for (int i = 0; i <= p; ++i) {
    double Pp = 1.0;
    if (i != 0 && i != p) {
      double a = 1.0, b = x[i];
      for (int k = 2; k <= p; ++k) {
        const double c = ((2.0 * k - 1.0) * x[i] * b - (k - 1.0) * a) / k;
        a = b;
        b = c;
      }
      Pp = b;
    }
    w[i] = 2.0 / (p * (p + 1.0) * Pp * Pp);
  }
}

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

}  // namespace

using namespace dgpf;

extern "C" dg_status dg_rhs_noalloc(const dg_mesh *mesh, int p, const dg_eos *eos, double Gamma, double eps,
                                    const dg_opts *opts, const double *w, double *L, void *stream) {
  // Arguments (same rules as dg_create / dg_rhs); nothing touches the GPU before they pass.
  if (!mesh || !eos || !w || !L || w == L) return DG_ERR_ARG;
  if (mesh->dim != 1 && mesh->dim != 2) return DG_ERR_ARG;
  if (mesh->elem != DG_ELEM_QUAD) return mesh->elem == DG_ELEM_TRI ? DG_ERR_UNSUPPORTED : DG_ERR_ARG;
  if (p < 1 || p > 5) return DG_ERR_UNSUPPORTED;
  if (mesh->nx < 1 || mesh->ny < 1 || (mesh->dim == 1 && mesh->ny != 1)) return DG_ERR_ARG;
  if (!(mesh->x1 > mesh->x0) || (mesh->dim == 2 && !(mesh->y1 > mesh->y0))) return DG_ERR_ARG;
  for (int f = 0; f < 4; ++f)
    if (mesh->bc[f] < DG_BC_PERIODIC || mesh->bc[f] > DG_BC_SLIP) return DG_ERR_ARG;
  if ((mesh->bc[0] == DG_BC_PERIODIC) != (mesh->bc[1] == DG_BC_PERIODIC) ||
      (mesh->dim == 2 && (mesh->bc[2] == DG_BC_PERIODIC) != (mesh->bc[3] == DG_BC_PERIODIC)))
    return DG_ERR_ARG;
  for (int l = 0; l < 2; ++l)
    if (!(eos->gamma[l] > 1.0) || !(eos->rho0[l] > 0.0) || eos->mu[l] < 0.0) return DG_ERR_ARG;
  if (!(Gamma >= 0.0) || !(eps >= 0.0)) return DG_ERR_ARG;
  const double c_ip = (opts && opts->c_ip > 0.0) ? opts->c_ip : 1.0;
  const bool viscous = opts && opts->viscous, st = opts && opts->surface_tension, grav = opts && opts->gravity;
  if (opts && opts->prec != DG_FP64) return DG_ERR_UNSUPPORTED;
  KernelSet ks;
  if (!kernels_fp64(p, mesh->dim, viscous, st, &ks)) return DG_ERR_UNSUPPORTED;

  const int dim = mesh->dim, P1 = p + 1, Np = dim == 2 ? P1 * P1 : P1;
  const long long E = (long long)mesh->nx * mesh->ny;
  const long long N = E * Np;
  const int NFK = 2 * dim * (dim == 2 ? P1 : 1);
  const OpsLayout lay{P1, Np};
  // scratch: status word | operator table | volume part (7 N) | face traces (nt E NFK)
  const size_t off_ops = 256;
  const size_t off_rvol = off_ops + align256(sizeof(double) * lay.size());
  const size_t off_tr = off_rvol + align256(sizeof(double) * 7 * (size_t)N);
  const size_t need = off_tr + sizeof(double) * (size_t)ks.nt * (size_t)E * NFK;
  if (need > (size_t)DG_NOALLOC_SCRATCH_BYTES) return DG_ERR_ARG;  // too large for the fixed scratch

  unsigned char *base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return DG_ERR_CUDA;
  double *d_ops = reinterpret_cast<double *>(base + off_ops);
  double *d_rvol = reinterpret_cast<double *>(base + off_rvol);
  double *d_tr = reinterpret_cast<double *>(base + off_tr);
  unsigned *d_status = reinterpret_cast<unsigned *>(base);

  // Operator table on the host stack (p <= 5: at most 198 doubles).
  double xi[6], wt[6], lam[6], D[36], ops[4 * 36 + 3 * 6 + 36];
  gll(p, xi, wt);
  for (int j = 0; j < P1; ++j) {
    lam[j] = 1.0;
    for (int k = 0; k < P1; ++k)
      if (k != j) lam[j] /= (xi[j] - xi[k]);
  }
  for (int a = 0; a < P1; ++a) {
    double diag = 0.0;
    for (int b = 0; b < P1; ++b) {
      if (b == a) continue;
      D[a * P1 + b] = (lam[b] / lam[a]) / (xi[a] - xi[b]);
      diag -= D[a * P1 + b];
    }
    D[a * P1 + a] = diag;
  }
  const double hx = (mesh->x1 - mesh->x0) / mesh->nx;
  const double hy = dim == 2 ? (mesh->y1 - mesh->y0) / mesh->ny : 1.0;
  const double J = dim == 2 ? 0.25 * hx * hy : 0.5 * hx;
  for (int a = 0; a < P1; ++a)
    for (int b = 0; b < P1; ++b) {
      ops[lay.Dx() + a * P1 + b] = (2.0 / hx) * D[a * P1 + b];
      ops[lay.Dy() + a * P1 + b] = (2.0 / hy) * D[a * P1 + b];
      const double dh = wt[b] * D[b * P1 + a] / wt[a];
      ops[lay.Dhx() + a * P1 + b] = (2.0 / hx) * dh;
      ops[lay.Dhy() + a * P1 + b] = (2.0 / hy) * dh;
    }
  for (int a = 0; a < P1; ++a) ops[lay.wt() + a] = wt[a];
  for (int a = 0; a < Np; ++a) ops[lay.invM() + a] = 1.0 / ((dim == 2 ? wt[a % P1] * wt[a / P1] : wt[a]) * J);
  for (int k = 0; k < P1; ++k) {
    ops[lay.wfx() + k] = dim == 2 ? wt[k] * 0.5 * hy : 1.0;
    ops[lay.wfy() + k] = dim == 2 ? wt[k] * 0.5 * hx : 1.0;
  }

  Params q{};
  q.nx = mesh->nx;
  q.ny = mesh->ny;
  q.E = (int)E;
  q.N = (int)N;
  for (int f = 0; f < 4; ++f) q.bc[f] = mesh->bc[f];
  q.C1 = eos->gamma[0] * eos->pinf[0] / (eos->gamma[0] - 1.0);
  q.C2 = eos->gamma[1] * eos->pinf[1] / (eos->gamma[1] - 1.0);
  q.g1 = 1.0 / (eos->gamma[0] - 1.0);
  q.g2 = 1.0 / (eos->gamma[1] - 1.0);
  q.Bp = eos->gamma[0] / (eos->gamma[0] - 1.0) - eos->gamma[1] / (eos->gamma[1] - 1.0);
  q.dC = q.C1 - q.C2;
  q.rho01 = eos->rho0[0];
  q.rho02 = eos->rho0[1];
  q.drho0 = eos->rho0[0] - eos->rho0[1];
  q.mu1 = eos->mu[0];
  q.mu2 = eos->mu[1];
  q.sigma = eos->sigma;
  q.gx = eos->g[0];
  q.gy = eos->g[1];
  q.Gamma = Gamma;
  q.eps = eps;
  q.eta_x = c_ip * P1 * P1 / hx;
  q.eta_y = c_ip * P1 * P1 / hy;
  q.gravity = grav ? 1 : 0;
  q.check_finite = 0;  // no context to report it through
  q.ops = d_ops;
  q.status = d_status;

  cudaStream_t s = (cudaStream_t)stream;
  // The table comes from pageable host memory: the copy call returns only
  // after the source has been read, so the stack buffer may go out of scope.
  cudaError_t e = cudaMemcpyAsync(d_ops, ops, sizeof(double) * lay.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = ks.volume(q, w, d_rvol, d_tr, s);
  if (e == cudaSuccess) e = ks.surface(q, MODE_RHS, 0.0, w, w, d_rvol, d_tr, L, s);
  return e == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}
