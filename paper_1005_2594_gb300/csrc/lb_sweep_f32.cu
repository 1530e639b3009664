// lb_sweep_f32.cu -- the lattice sweep (lb_sweep.cuh) for FP32 storage.
#include "lb_sweep.cuh"

namespace bl {

void launch_lb_step_f32(const LatticeView &lv, int par, const WallAcc &wa, cudaStream_t st) {
  launch_lb_typed<float>(lv, par, wa, st);
}

void lb_rows_grids_f32(int out[8]) { rows_grids<float>(out); }

}  // namespace bl
