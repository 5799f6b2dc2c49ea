// Level-set re-initialisation kernels (dg_reinit.cuh) of orders 1..5, 1D and 2D.
#include "dg_reinit.cuh"

namespace dgpf {

template <int P, int DIM>
static ReinitKernels make_ri() {
  return ReinitKernels{&launch_ri_sign<P, DIM>, &launch_ri_volume<P, DIM>, &launch_ri_surface<P, DIM>,
                       Geom<P, DIM, false, false>::NFK};
}

template <int P>
static bool ri_p(int dim, ReinitKernels *out) {
  if (dim == 1) *out = make_ri<P, 1>();
  else if (dim == 2) *out = make_ri<P, 2>();
  else return false;
  return true;
}

bool reinit_kernels(int p, int dim, ReinitKernels *out) {
  switch (p) {
    case 1: return ri_p<1>(dim, out);
    case 2: return ri_p<2>(dim, out);
    case 3: return ri_p<3>(dim, out);
    case 4: return ri_p<4>(dim, out);
    case 5: return ri_p<5>(dim, out);
    default: return false;
  }
}

}  // namespace dgpf
