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
// The problem is validated and its operator table and parameters are built by
// the same host code as dg_create (dg_host.h); the table reaches the device as
// a kernel argument (no host-to-device copy).
#include <cuda_runtime.h>

#include <mutex>

#include "dg_common.cuh"
#include "dg_host.h"
#include "dgpf.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[DG_NOALLOC_SCRATCH_BYTES];

namespace {

using namespace dgpf;

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_addr[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// The largest operator table (p = 5, 2D).
constexpr int kMaxOps = 4 * HOST_MAXP1 * HOST_MAXP1 + 3 * HOST_MAXP1 + HOST_MAXP1 * HOST_MAXP1;
struct OpsArg {
  double v[kMaxOps];
};

// Writes the operator table (passed by value) into the scratch and clears the
// status word.  One block.
__global__ void k_noalloc_setup(OpsArg ops, int n, double *__restrict__ dst, unsigned *__restrict__ status) {
  for (int t = threadIdx.x; t < n; t += blockDim.x) dst[t] = ops.v[t];
  if (threadIdx.x == 0) *status = 0u;
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

extern "C" dg_status dg_rhs_noalloc(const dg_mesh *mesh, int p, const dg_eos *eos, double Gamma, double eps,
                                    const dg_opts *opts, const double *w, double *L, void *stream) {
  // Arguments: the rules of dg_create and dg_rhs; nothing touches the GPU before they pass.
  if (!w || !L || w == L) return DG_ERR_ARG;
  dg_status code;
  if (check_problem(mesh, p, eos, Gamma, eps, &code)) return code;
  const dg_opts o = normalised_opts(opts);
  if (o.prec != DG_FP64) return o.prec == DG_FP32_BULK ? DG_ERR_UNSUPPORTED : DG_ERR_ARG;
  if (o.grad_lift != 0 && o.grad_lift != 1) return DG_ERR_ARG;
  KernelSet ks;
  if (!kernels_fp64(p, mesh->dim, o.viscous != 0, o.surface_tension != 0, &ks)) return DG_ERR_UNSUPPORTED;

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

  const double hx = (mesh->x1 - mesh->x0) / mesh->nx;
  const double hy = dim == 2 ? (mesh->y1 - mesh->y0) / mesh->ny : 1.0;
  OpsArg ops;
  build_ops_into(dim, p, hx, hy, ops.v);
  Params q = make_params(mesh, p, eos, Gamma, eps, o, hx, hy);
  q.check_finite = 0;  // no context to report it through
  q.ops = d_ops;
  q.status = d_status;

  cudaStream_t s = (cudaStream_t)stream;
  k_noalloc_setup<<<1, 128, 0, s>>>(ops, lay.size(), d_ops, d_status);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = ks.volume(q, w, d_rvol, d_tr, s);
  if (e == cudaSuccess) e = ks.surface(q, MODE_RHS, 0.0, w, w, d_rvol, d_tr, L, s);
  return e == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}
