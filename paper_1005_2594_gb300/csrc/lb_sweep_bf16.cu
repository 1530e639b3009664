// lb_sweep_bf16.cu -- the lattice sweep (lb_sweep.cuh) for BF16 storage.
#include "lb_sweep.cuh"

namespace bl {

void launch_lb_step_bf16(const LatticeView &lv, int par, const WallAcc &wa, cudaStream_t st) {
  launch_lb_typed<__nv_bfloat16>(lv, par, wa, st);
}

void lb_rows_grids_bf16(int out[8]) { rows_grids<__nv_bfloat16>(out); }

}  // namespace bl
