// Kinematic-mode kernels (dg_kin.cuh) of orders 1..5.
#include "dg_kin.cuh"

namespace dgpf {

bool kin_kernels(int p, KinKernels *out) {
  switch (p) {
    case 1: *out = {&launch_kin_stage<1>, &launch_kin_velocity_table<1>}; return true;
    case 2: *out = {&launch_kin_stage<2>, &launch_kin_velocity_table<2>}; return true;
    case 3: *out = {&launch_kin_stage<3>, &launch_kin_velocity_table<3>}; return true;
    case 4: *out = {&launch_kin_stage<4>, &launch_kin_velocity_table<4>}; return true;
    case 5: *out = {&launch_kin_stage<5>, &launch_kin_velocity_table<5>}; return true;
    default: return false;
  }
}

// Sets the time base read by the kinematic kernels of a captured sequence.
__global__ void k_kin_set_time(double *t0, double t) { *t0 = t; }

}  // namespace dgpf
