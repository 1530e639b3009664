// lb_sweep_f16.cu -- the lattice sweep (lb_sweep.cuh) for FP16 storage.
#include "lb_sweep.cuh"

namespace bl {

void launch_lb_step_f16(const LatticeView &lv, int par, const WallAcc &wa, cudaStream_t st) {
  launch_lb_typed<__half>(lv, par, wa, st);
}

void lb_rows_grids_f16(int out[8]) { rows_grids<__half>(out); }

}  // namespace bl
