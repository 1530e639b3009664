// lb_kernels.cu -- the lattice sweep of the coupled step and the lattice-side
// helper kernels.
//
// The sweep fuses, per node and per time step (arXiv:1005.2594, Sec. II):
//   * moments rho, j and the Guo-forced velocity u = (j + rho g / 2) / rho,
//   * BGK collision (Eq. col) with the third-order equilibrium (Eq. neq),
//   * advection (Eq. adv) in the AA pattern on one buffer,
//   * mid-link bounce-back (Eq. lbe-bb); on wall links with the moving-wall
//     term C (Eqs. c, lbe-bb-corr) and the momentum exchange (Eq. deltap)
//     into the wall's counter.
//
// AA pattern.  Slot r of node n sits at r * N + n.  An even step reads node
// n's populations from its own slots [r][n] and writes the post-collision
// value of direction r to [rbar][n]; an odd step reads [rbar][n - c_r] and
// writes [r][n + c_r].  A population that meets a solid neighbour is written,
// with C added, to the slot where the next step reads the opposite direction
// of the same node: [r][n + c_r] in an even step, [rbar][n] in an odd one.
// Every fluid node reads and writes its own 19 slots only, so the sweep is
// race-free in place.  Populations are stored shifted, f~ = f - alpha rho_bar.
//
// Cells.  A population that meets a cell node is bounced here without the
// moving-boundary term: the cell's velocity of the half step is not known
// yet.  The sweep records the node's density; the cell kernels then sum the
// cell's link momenta over its link list, solve for the half-step velocity
// and add C to each of its bounced populations (reading Q3, implicit
// coupling).
// Walls move at a known velocity: their links get C here, and the wall's
// momentum is summed per warp (constant part 2 alpha_r rho_bar c_r as exact
// integers) before one atomic per wall and component.
//
// Geometry pass.  After every change of the owner map one lattice-wide pass
// (k_geometry) writes each fluid node's neighbour word -- so the sweep reads
// one word per node instead of 18 neighbour owners -- and, at each cell node,
// appends the cell's bounce links and sums its contact links.
#include "bl_internal.cuh"

namespace bl {

// blocks of 128 threads resident per SM: 8 caps the sweep at 64 registers
#ifndef BL_LB_MINB
#define BL_LB_MINB 8
#endif

// warp-level sum of the wall momenta, one atomic per wall and component
// (all lanes of the warp call it)
__device__ __forceinline__ void flush_wall_momentum(const WallAcc &wa, int &wkey, float (&wF)[3], int (&wK)[3]) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  unsigned pending = __ballot_sync(FULL, wkey >= 0);
  while (pending) {
    const int leader = __ffs(pending) - 1;
    const int lk = __shfl_sync(FULL, wkey, leader);
    const bool mine = wkey == lk;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float vs = warp_sum(mine ? wF[k] : 0.f);
      const int is = __reduce_add_sync(FULL, mine ? wK[k] : 0);
      if (lane == leader) {
        atomicAdd(&wa.F[3 * lk + k], (double)vs);
        atomicAdd((unsigned long long *)&wa.K[3 * lk + k], (unsigned long long)(long long)is);
      }
    }
    pending &= ~__ballot_sync(FULL, mine);
    if (mine) wkey = -1;
  }
}

// index of the slot from which node n reads direction r in a step of parity
// PAR (xo, yo, zo: coordinates of its 3 x 3 x 3 neighbourhood, y and z
// pre-multiplied by their strides)
template <int PAR>
__device__ __forceinline__ unsigned src_slot(int r, unsigned N, unsigned n, const unsigned xo[3], const unsigned yo[3],
                                             const unsigned zo[3]) {
  using D = D3Q19;
  if (PAR == 0 || r == 0) return (unsigned)r * N + n;
  return (unsigned)D::opp(r) * N + xo[1 - D::cx(r)] + yo[1 - D::cy(r)] + zo[1 - D::cz(r)];
}

// One fluid node of the sweep: moments, collision, streaming with
// bounce-back and the wall momentum.  load(r, slot) gives the incoming
// population of direction r (from the slot src_slot names).
// FORCE: a body force is set (Guo forcing); TAU1: tau = 1, where the
// relaxation gives the equilibrium itself
template <class S, int PAR, bool FORCE, bool TAU1, class Load>
__device__ __forceinline__ void node_update(const LatticeView &lv, const WallAcc &wa, int *status, unsigned n,
                                            const unsigned xo[3], const unsigned yo[3], const unsigned zo[3],
                                            uint32_t nbw, Load load, int &wkey, float (&wF)[3], int (&wK)[3]) {
  using D = D3Q19;
  const unsigned N = lv.N;
  S *pop = reinterpret_cast<S *>(lv.pop);
  if (nbw & NB_FLUID) {
    // neighbour classes from the geometry pass: solid = any non-fluid node;
    // the wall subset is looked up only next to a wall
    const unsigned solid = nbw & NB_SOLID;
    unsigned wall = 0;
    if (nbw & NB_WALL) {
      sfor<1, Q>([&](auto R) {
        constexpr int r = decltype(R)::value;
        if (solid & (1u << r)) {
          const unsigned nb = xo[1 + D::cx(r)] + yo[1 + D::cy(r)] + zo[1 + D::cz(r)];
          wall |= (lv.owner[nb] <= -2 ? 1u : 0u) << r;
        }
      });
    }
    // incoming populations of this node (layout of the step's parity)
    float f[Q];
    sfor<0, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      unsigned src;
      if constexpr (PAR == 0 || r == 0) {
        src = (unsigned)r * N + n;
      } else {
        src = (unsigned)D::opp(r) * N + xo[1 - D::cx(r)] + yo[1 - D::cy(r)] + zo[1 - D::cz(r)];
      }
      f[r] = load(r, src);
    });
    // moments (shifted: rho = rho_bar + sum f~, j = sum f~ c)
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
    sfor<0, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      drho += f[r];
      if constexpr (D::cx(r) != 0) jx += D::cx(r) * f[r];
      if constexpr (D::cy(r) != 0) jy += D::cy(r) * f[r];
      if constexpr (D::cz(r) != 0) jz += D::cz(r) * f[r];
    });
    const float rho = lv.rho0 + drho;
    const float inv = 1.0f / rho;
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    if constexpr (FORCE) {
      Fx = rho * lv.g[0];
      Fy = rho * lv.g[1];
      Fz = rho * lv.g[2];
    }
    const float ux = (jx + 0.5f * Fx) * inv, uy = (jy + 0.5f * Fy) * inv, uz = (jz + 0.5f * Fz) * inv;
    const float uu = ux * ux + uy * uy + uz * uz;
    if (!(rho > 0.f) || !(uu < 0.09f)) atomicOr(status, ST_UNSTABLE);
    const float om = lv.omega;
    const float src_w = 1.0f - 0.5f * om;
    const float uF = ux * Fx + uy * Fy + uz * Fz;
    // relaxation toward the shifted equilibrium w (drho + rho t); rho t is
    // taken as rho_bar t + drho t, which keeps the small deviation exact in
    // FP32; the Guo source with cu = c.u, cF = c.F
    auto relax = [&](float fr, float w, float t, float cu, float cF) {
      const float feq = w * (drho + fmaf(drho, t, lv.rho0 * t));
      float fs = TAU1 ? feq : fr - om * (fr - feq);
      if constexpr (FORCE) fs += src_w * w * (3.0f * (cF - uF) + 9.0f * cu * cF);
      return fs;
    };
    // third-order equilibrium in pairs r, rbar = r + 1 (c_rbar = -c_r):
    // t = E + O and E - O with the even part E = 4.5 cu^2 - 1.5 uu and the
    // odd part O = cu (3 + 4.5 cu^2 - 4.5 uu)
    const float a = 3.0f - 4.5f * uu, b = 1.5f * uu;
    f[0] = relax(f[0], 12.0f / 36.0f, -b, 0.f, 0.f);
    sfor<0, 9>([&](auto P) {
      constexpr int r = 2 * decltype(P)::value + 1, rb = r + 1;
      constexpr float w = D::m(r) / 36.0f;
      float cu = 0.f, cF = 0.f;
      if constexpr (D::cx(r) != 0) cu += D::cx(r) * ux;
      if constexpr (D::cy(r) != 0) cu += D::cy(r) * uy;
      if constexpr (D::cz(r) != 0) cu += D::cz(r) * uz;
      if constexpr (FORCE) cF = D::cx(r) * Fx + D::cy(r) * Fy + D::cz(r) * Fz;
      const float q = 4.5f * cu * cu;
      const float E = q - b, O = cu * (a + q);
      f[r] = relax(f[r], w, E + O, cu, cF);
      f[rb] = relax(f[rb], w, E - O, -cu, -cF);
    });
    Store<S>::st(pop + n, f[0]);
    if (wall) {
      // links into a wall (next to a wall only): the moving-wall term C for
      // the population returning along rbar, 6 alpha_rbar rho c_rbar . v_wall,
      // and the momentum the wall receives
      sfor<1, Q>([&](auto R) {
        constexpr int r = decltype(R)::value;
        if (wall & (1u << r)) {
          const unsigned nb = xo[1 + D::cx(r)] + yo[1 + D::cy(r)] + zo[1 + D::cz(r)];
          const int w = -2 - lv.owner[nb];
          const float C = -(D::m(r) / 6.0f) * rho *
                          (D::cx(r) * lv.wall_vel[w][0] + D::cy(r) * lv.wall_vel[w][1] + D::cz(r) * lv.wall_vel[w][2]);
          const float dp = 2.0f * f[r] + C;
          if (wkey != w && wkey >= 0) {
            // a node touching two different walls: flush the first one directly
            for (int k = 0; k < 3; ++k) {
              atomicAdd(&wa.F[3 * wkey + k], (double)wF[k]);
              atomicAdd((unsigned long long *)&wa.K[3 * wkey + k], (unsigned long long)(long long)wK[k]);
              wF[k] = 0.f;
              wK[k] = 0;
            }
          }
          wkey = w;
          wF[0] += dp * D::cx(r);
          wF[1] += dp * D::cy(r);
          wF[2] += dp * D::cz(r);
          wK[0] += D::m(r) * D::cx(r);
          wK[1] += D::m(r) * D::cy(r);
          wK[2] += D::m(r) * D::cz(r);
          f[r] += C;
        }
      });
    }
    // streaming, or bounce-back into the slot where the next step reads
    // direction rbar where the neighbour is solid: one store per direction,
    // its slot chosen without a branch (so that a warp mixing open and
    // boundary nodes writes each row of slots with one instruction)
    //   parity 0: open -> [rbar][n],       solid -> [r][n + c_r]
    //   parity 1: open -> [r][n + c_r],    solid -> [rbar][n]
    sfor<1, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      constexpr int rb = D::opp(r);
      const unsigned nb = xo[1 + D::cx(r)] + yo[1 + D::cy(r)] + zo[1 + D::cz(r)];
      const bool sol = (solid >> r) & 1u;
      const unsigned dst = (sol != (PAR == 1)) ? (unsigned)r * N + nb : (unsigned)rb * N + n;
      Store<S>::st(pop + dst, f[r]);
    });
    if (nbw & NB_CELL) lv.rho_b[n] = rho;
  }
}

template <class S, int PAR, bool FORCE, bool TAU1>
__global__ void __launch_bounds__(128, BL_LB_MINB) k_lb_step(LatticeView lv, WallAcc wa, int *status) {
  const int nx = lv.nx, ny = lv.ny;
  const int x0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  const bool valid = x0 < nx;
  const int x = valid ? x0 : nx - 1;
  const unsigned nxy = (unsigned)nx * (unsigned)ny;
  const unsigned n = (unsigned)x + (unsigned)nx * (unsigned)y + nxy * (unsigned)z;
  // coordinates of the 3 x 3 x 3 neighbourhood, periodic wrap on every axis
  // (a walled axis has wall layers at both ends, never crossed by a link)
  const unsigned xo[3] = {(unsigned)(x == 0 ? nx - 1 : x - 1), (unsigned)x, (unsigned)(x == nx - 1 ? 0 : x + 1)};
  const unsigned yo[3] = {(unsigned)(y == 0 ? ny - 1 : y - 1) * nx, (unsigned)y * nx,
                          (unsigned)(y == ny - 1 ? 0 : y + 1) * nx};
  const unsigned zo[3] = {(unsigned)(z == 0 ? lv.nz - 1 : z - 1) * nxy, (unsigned)z * nxy,
                          (unsigned)(z == lv.nz - 1 ? 0 : z + 1) * nxy};
  const S *pop = reinterpret_cast<const S *>(lv.pop);
  const uint32_t nbw = valid ? lv.nbm[n] : 0u;
  // wall momentum of this thread: wall id, variable part, constant-part integers
  int wkey = -1;
  float wF[3] = {0.f, 0.f, 0.f};
  int wK[3] = {0, 0, 0};
  if (nbw & NB_FLUID)
    node_update<S, PAR, FORCE, TAU1>(lv, wa, status, n, xo, yo, zo, nbw,
                                     [&](int, unsigned slot) { return Store<S>::ld(pop + slot); }, wkey, wF, wK);
  flush_wall_momentum(wa, wkey, wF, wK);
}

// The FP32 sweep as a software pipeline along z: a block of 128 threads takes
// a row segment and ZC consecutive z planes; while a node is collided,
// the populations of the next PIPE_ST - 1 nodes above it are on their way
// into shared memory (asynchronous 4-byte copies, one group per node).  The
// neighbour word of a node is loaded just before its copies are issued;
// solid nodes copy nothing.
#ifndef BL_PIPE_ST
#define BL_PIPE_ST 2
#endif
constexpr int PIPE_ST = BL_PIPE_ST;

__device__ __forceinline__ void cp_async4(void *dst_smem, const void *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int G>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(G) : "memory");
}

template <int PAR, bool FORCE, bool TAU1, int ZC>
__global__ void __launch_bounds__(128, BL_LB_MINB) k_lb_step_pipe(LatticeView lv, WallAcc wa, int *status) {
  __shared__ float stage[PIPE_ST][Q][128];
  const int nx = lv.nx, ny = lv.ny, nz = lv.nz;
  const int tx = threadIdx.x;
  const int x0 = blockIdx.x * blockDim.x + tx;
  const int y = blockIdx.y;
  const int zb = blockIdx.z * ZC, ze = min(zb + ZC, nz);
  const bool valid = x0 < nx;
  const int x = valid ? x0 : nx - 1;
  const unsigned N = lv.N;
  const unsigned nxy = (unsigned)nx * (unsigned)ny;
  const unsigned xo[3] = {(unsigned)(x == 0 ? nx - 1 : x - 1), (unsigned)x, (unsigned)(x == nx - 1 ? 0 : x + 1)};
  const unsigned yo[3] = {(unsigned)(y == 0 ? ny - 1 : y - 1) * nx, (unsigned)y * nx,
                          (unsigned)(y == ny - 1 ? 0 : y + 1) * nx};
  const unsigned rowb = (unsigned)x + (unsigned)nx * (unsigned)y;
  const float *pop = reinterpret_cast<const float *>(lv.pop);
  auto zoff = [&](int z, unsigned zo[3]) {
    zo[0] = (unsigned)(z == 0 ? nz - 1 : z - 1) * nxy;
    zo[1] = (unsigned)z * nxy;
    zo[2] = (unsigned)(z == nz - 1 ? 0 : z + 1) * nxy;
  };
  // neighbour word of node z, and its copies into stage buffer b when fluid
  auto issue = [&](int z, int b) -> uint32_t {
    if (!valid || z >= ze) return 0u;
    unsigned zo[3];
    zoff(z, zo);
    const unsigned n = rowb + zo[1];
    const uint32_t w = lv.nbm[n];
    if (w & NB_FLUID)
      sfor<0, Q>([&](auto R) {
        constexpr int r = decltype(R)::value;
        cp_async4(&stage[b][r][tx], pop + src_slot<PAR>(r, N, n, xo, yo, zo));
      });
    return w;
  };
  int wkey = -1;
  float wF[3] = {0.f, 0.f, 0.f};
  int wK[3] = {0, 0, 0};
  uint32_t w[PIPE_ST];  // neighbour words of the nodes in flight, oldest first
#pragma unroll
  for (int k = 0; k < PIPE_ST - 1; ++k) {
    w[k] = issue(zb + k, k);
    cp_async_commit();
  }
  for (int z = zb; z < ze; ++z) {
    const int i = z - zb;
    w[PIPE_ST - 1] = issue(z + PIPE_ST - 1, (i + PIPE_ST - 1) % PIPE_ST);
    cp_async_commit();
    cp_async_wait<PIPE_ST - 1>();  // the copies of node z have landed
    const int b = i % PIPE_ST;
    if (w[0] & NB_FLUID) {
      unsigned zo[3];
      zoff(z, zo);
      node_update<float, PAR, FORCE, TAU1>(lv, wa, status, rowb + zo[1], xo, yo, zo, w[0],
                                           [&](int r, unsigned) { return stage[b][r][tx]; }, wkey, wF, wK);
    }
#pragma unroll
    for (int k = 0; k < PIPE_ST - 1; ++k) w[k] = w[k + 1];
  }
  cp_async_wait<0>();
  flush_wall_momentum(wa, wkey, wF, wK);
}

// The sweep fed by bulk asynchronous copies (TMA, untiled): a block of
// 128 threads takes a row segment of up to 128 nodes and ZC consecutive z
// planes.  For each plane one thread copies the 19 source row segments and
// the row of neighbour words into shared memory with cp.async.bulk, TS - 1
// planes ahead of the plane being collided, each stage completing on its
// mbarrier.  Parity 0 reads row (y, z) of array r; parity 1 reads row
// (y - c_y, z - c_z) of array rbar, element x - c_x: from shared memory when
// it lies in the segment (the whole row when the segment is the whole
// periodic row), else directly from global memory.  Needs 16-byte aligned
// rows: nx % 4 == 0 for FP32 storage, nx % 8 == 0 for BF16 / FP16; every
// wait is bounded (ST_BARRIER after ~2^26 polls).

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned phase) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return done != 0;
}
// bounded wait: false if the copies did not land within the limit
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned phase) {
  for (int it = 0; it < (1 << 26); ++it)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

template <class S, int PAR, bool FORCE, bool TAU1, int ZC, int TS>
__global__ void __launch_bounds__(128, 6) k_lb_step_bulk(LatticeView lv, WallAcc wa, int *status) {
  using D = D3Q19;
  __shared__ alignas(128) S sb[TS][Q][128];        // [stage][array][x]
  __shared__ alignas(128) uint32_t sw[TS][128];    // [stage][x] neighbour words
  __shared__ alignas(8) unsigned long long bar[TS];
  __shared__ int s_ok;
  const int nx = lv.nx, ny = lv.ny, nz = lv.nz;
  const int tx = threadIdx.x;
  const int x0 = blockIdx.x * 128;
  const int W = min(128, nx - x0);  // segment width, a multiple of 4
  const bool whole = W == nx;       // the segment is the whole row
  const int y = blockIdx.y;
  const int zb = blockIdx.z * ZC, ze = min(zb + ZC, nz);
  const bool valid = tx < W;
  const int x = x0 + (valid ? tx : W - 1);
  const unsigned N = lv.N;
  const unsigned nxy = (unsigned)nx * (unsigned)ny;
  const unsigned xo[3] = {(unsigned)(x == 0 ? nx - 1 : x - 1), (unsigned)x, (unsigned)(x == nx - 1 ? 0 : x + 1)};
  const unsigned yo[3] = {(unsigned)(y == 0 ? ny - 1 : y - 1) * nx, (unsigned)y * nx,
                          (unsigned)(y == ny - 1 ? 0 : y + 1) * nx};
  const S *pop = reinterpret_cast<const S *>(lv.pop);
  auto zoff = [&](int z, unsigned zo[3]) {
    zo[0] = (unsigned)(z == 0 ? nz - 1 : z - 1) * nxy;
    zo[1] = (unsigned)z * nxy;
    zo[2] = (unsigned)(z == nz - 1 ? 0 : z + 1) * nxy;
  };
  // one thread: the copies of plane z into stage s
  auto issue = [&](int z, int s) {
    if (z >= ze) return;
    unsigned zo[3];
    zoff(z, zo);
    const unsigned bytes = (unsigned)W * (unsigned)sizeof(S);
    mbar_expect_tx(&bar[s], Q * bytes + (unsigned)W * 4u);
    sfor<0, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      unsigned row;
      if constexpr (PAR == 0 || r == 0) row = (unsigned)r * N + yo[1] + zo[1];
      else row = (unsigned)D::opp(r) * N + yo[1 - D::cy(r)] + zo[1 - D::cz(r)];
      bulk_g2s(&sb[s][r][0], pop + row + (unsigned)x0, bytes, &bar[s]);
    });
    bulk_g2s(&sw[s][0], lv.nbm + yo[1] + zo[1] + (unsigned)x0, (unsigned)W * 4u, &bar[s]);
  };
  if (tx == 0) {
    for (int k = 0; k < TS; ++k) mbar_init(&bar[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_ok = 1;
  }
  __syncthreads();
  if (tx == 0)
    for (int k = 0; k < TS - 1; ++k) issue(zb + k, k);
  int wkey = -1;
  float wF[3] = {0.f, 0.f, 0.f};
  int wK[3] = {0, 0, 0};
  int z = zb;
  for (; z < ze; ++z) {
    const int i = z - zb, s = i % TS;
    if (tx == 0) issue(z + TS - 1, (i + TS - 1) % TS);  // that stage was freed by the last barrier
    if (!mbar_wait(&bar[s], (unsigned)(i / TS) & 1u)) {
      atomicOr(status, ST_BARRIER);
      s_ok = 0;
    }
    __syncthreads();
    if (!s_ok) break;
    const uint32_t w = valid ? sw[s][tx] : 0u;
    if (w & NB_FLUID) {
      unsigned zo[3];
      zoff(z, zo);
      node_update<S, PAR, FORCE, TAU1>(
          lv, wa, status, (unsigned)x + yo[1] + zo[1], xo, yo, zo, w,
          [&](int r, unsigned slot) -> float {
            if (PAR == 0 || r == 0) return Store<S>::ld(&sb[s][r][tx]);
            int j = tx - D::cx(r);
            if (whole) j = j < 0 ? j + W : (j >= W ? j - W : j);
            return (j >= 0 && j < W) ? Store<S>::ld(&sb[s][r][j]) : Store<S>::ld(pop + slot);
          },
          wkey, wF, wK);
    }
    __syncthreads();  // stage s is read: free for refill
  }
  if (z < ze && tx == 0) {
    // gave up: let the copies still in flight land before the block exits
    for (int k = 0; k < TS; ++k) mbar_wait(&bar[k], 0u), mbar_wait(&bar[k], 1u);
  }
  flush_wall_momentum(wa, wkey, wF, wK);
}

// ---------------------------------------------------------------------------
// geometry pass over the owner map (one thread per node, 128 along x)
//
//   fluid node  -> neighbour word (NB_* bits)
//   cell node x of cell p, neighbour x + c_r fluid -> bounce link of p: the
//                  fluid node y = x + c_r streams direction rbar into p
//   cell node x of cell p, neighbour x + c_r another cell or a wall -> contact
//                  link (Eqs. deltapppp, deltapppm): its constant momentum
//                  -2 alpha_r rho_bar c_r goes into p's exact integer sums
//                  cK = sum m_r c_r, cIT = sum m_r dI x c_r, dI = x - rint(X_p)
//
// A warp appends its links cell by cell with one atomic on the cell's count,
// in direction order, so that the link kernels read consecutive nodes of one
// direction.  The counts start at zero (the claims kernel clears them).
__global__ void __launch_bounds__(128) k_geometry(LatticeView lv, PartView pv) {
  using D = D3Q19;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int nx = lv.nx, ny = lv.ny;
  const int x0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  const bool valid = x0 < nx;
  const int x = valid ? x0 : nx - 1;
  const unsigned nxy = (unsigned)nx * (unsigned)ny;
  const unsigned n = (unsigned)x + (unsigned)nx * (unsigned)y + nxy * (unsigned)z;
  const int xs[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};
  const int ys[3] = {y == 0 ? ny - 1 : y - 1, y, y == ny - 1 ? 0 : y + 1};
  const int zs[3] = {z == 0 ? lv.nz - 1 : z - 1, z, z == lv.nz - 1 ? 0 : z + 1};
  const int own = valid ? lv.owner[n] : -2;
  unsigned lmask = 0, cmask = 0;
  if (own >= FLUID) {
    unsigned solid = 0, wall = 0, same = 0;
    sfor<1, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      const unsigned nb = (unsigned)xs[1 + D::cx(r)] + (unsigned)nx * (unsigned)ys[1 + D::cy(r)] +
                          nxy * (unsigned)zs[1 + D::cz(r)];
      const int on = lv.owner[nb];
      solid |= (on != FLUID ? 1u : 0u) << r;
      wall |= (on <= -2 ? 1u : 0u) << r;
      same |= (on == own ? 1u : 0u) << r;
    });
    if (own == FLUID) {
      lv.nbm[n] = NB_FLUID | solid | (wall ? NB_WALL : 0u) | ((solid & ~wall) ? NB_CELL : 0u);
    } else {
      lv.nbm[n] = 0u;
      lmask = NB_SOLID & ~solid;  // fluid neighbours
      cmask = solid & ~same;      // other cells and walls
    }
  } else if (valid) {
    lv.nbm[n] = 0u;
  }
  if (pv.n == 0) return;  // no cell nodes: nothing to append (uniform per launch)

  // bounce links, one group of lanes per cell
  unsigned pend = __ballot_sync(FULL, lmask != 0u);
  while (pend) {
    const int leader = __ffs(pend) - 1;
    const int cell = __shfl_sync(FULL, own, leader);
    const bool mine = lmask != 0u && own == cell;
    const unsigned grp = __ballot_sync(FULL, mine);
    const int tot = __reduce_add_sync(FULL, mine ? __popc(lmask) : 0);
    int base = 0;
    if (lane == leader) base = atomicAdd(&pv.lk_count[cell], tot);
    base = __shfl_sync(FULL, base, leader);
    if (base + tot > pv.lk_cap && lane == leader) atomicOr(pv.status, ST_OVERFLOW);
    unsigned long long *lk = pv.lk + (size_t)cell * pv.lk_cap;
    const unsigned below = (1u << lane) - 1u;
    int run = base;
    sfor<1, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      const bool has = mine && ((lmask >> r) & 1u);
      const unsigned b = __ballot_sync(FULL, has);
      if (has) {
        const int pos = run + __popc(b & below);
        if (pos < pv.lk_cap)
          lk[pos] = pack_xyzr(xs[1 + D::cx(r)], ys[1 + D::cy(r)], zs[1 + D::cz(r)], D::opp(r));
      }
      run += __popc(b);
    });
    pend &= ~grp;
  }

  // contact links as exact integer sums
  int ci[6] = {0, 0, 0, 0, 0, 0};
  if (cmask) {
    const float4 k0 = pv.kin_next[3 * own], k1 = pv.kin_next[3 * own + 1], k2 = pv.kin_next[3 * own + 2];
    const int di[3] = {imin_image(x - (int)k0.w, nx, lv.per[0]), imin_image(y - (int)k1.w, ny, lv.per[1]),
                       imin_image(z - (int)k2.w, lv.nz, lv.per[2])};
    sfor<1, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      constexpr int m = D::m(r);
      if ((cmask >> r) & 1u) {
        ci[0] -= m * D::cx(r);
        ci[1] -= m * D::cy(r);
        ci[2] -= m * D::cz(r);
        ci[3] -= m * (di[1] * D::cz(r) - di[2] * D::cy(r));
        ci[4] -= m * (di[2] * D::cx(r) - di[0] * D::cz(r));
        ci[5] -= m * (di[0] * D::cy(r) - di[1] * D::cx(r));
      }
    });
  }
  pend = __ballot_sync(FULL, cmask != 0u);
  while (pend) {
    const int leader = __ffs(pend) - 1;
    const int cell = __shfl_sync(FULL, own, leader);
    const bool mine = cmask != 0u && own == cell;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int v = __reduce_add_sync(FULL, mine ? ci[k] : 0);
      if (lane == leader && v != 0) atomicAdd(k < 3 ? &pv.cK[3 * cell + k] : &pv.cIT[3 * cell + k - 3], v);
    }
    pend &= ~__ballot_sync(FULL, mine);
  }
}

// ---------------------------------------------------------------------------
// moments of the current populations (layout of parity par)

template <class S>
__global__ void k_fields(LatticeView lv, int par, double *rho_out, double *u_out, int32_t *owner_out) {
  using D = D3Q19;
  const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= lv.N) return;
  const int own = lv.owner[n];
  if (owner_out) owner_out[n] = own;
  if (own != FLUID) {
    if (rho_out) rho_out[n] = 0.0;
    if (u_out) u_out[3 * n] = u_out[3 * n + 1] = u_out[3 * n + 2] = 0.0;
    return;
  }
  const int nx = lv.nx, ny = lv.ny, nz = lv.nz;
  const int x = n % nx, y = (n / nx) % ny, z = n / ((unsigned)nx * ny);
  const S *pop = reinterpret_cast<const S *>(lv.pop);
  double drho = 0.0, j[3] = {0.0, 0.0, 0.0};
  for (int r = 0; r < Q; ++r) {
    unsigned src;
    if (par == 0 || r == 0) {
      src = (unsigned)r * lv.N + n;
    } else {
      const int xs = wrapi(x - D::cx(r), nx), ys = wrapi(y - D::cy(r), ny), zs = wrapi(z - D::cz(r), nz);
      src = (unsigned)D::opp(r) * lv.N + (unsigned)xs + (unsigned)nx * ((unsigned)ys + (unsigned)ny * zs);
    }
    const double v = Store<S>::ld(pop + src);
    drho += v;
    j[0] += v * D::cx(r);
    j[1] += v * D::cy(r);
    j[2] += v * D::cz(r);
  }
  const double rho = (double)lv.rho0 + drho;
  if (rho_out) rho_out[n] = rho;
  if (u_out)
    for (int k = 0; k < 3; ++k) u_out[3 * n + k] = (j[k] + 0.5 * rho * (double)lv.g[k]) / rho;
}

// node-major unshifted FP64 populations <-> storage (layout of parity par)
template <class S>
__global__ void k_pop_io(LatticeView lv, int par, double *host_layout, int to_storage) {
  using D = D3Q19;
  const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= lv.N) return;
  const bool fluid = lv.owner[n] == FLUID;
  const int nx = lv.nx, ny = lv.ny, nz = lv.nz;
  const int x = n % nx, y = (n / nx) % ny, z = n / ((unsigned)nx * ny);
  S *pop = reinterpret_cast<S *>(lv.pop);
  for (int r = 0; r < Q; ++r) {
    unsigned slot;
    if (par == 0 || r == 0) {
      slot = (unsigned)r * lv.N + n;
    } else {
      const int xs = wrapi(x - D::cx(r), nx), ys = wrapi(y - D::cy(r), ny), zs = wrapi(z - D::cz(r), nz);
      slot = (unsigned)D::opp(r) * lv.N + (unsigned)xs + (unsigned)nx * ((unsigned)ys + (unsigned)ny * zs);
    }
    const double shift = (double)lv.rho0 * D::m(r) / 36.0;
    if (to_storage) {
      if (fluid) Store<S>::st(pop + slot, (float)(host_layout[(size_t)n * Q + r] - shift));
    } else {
      host_layout[(size_t)n * Q + r] = fluid ? (double)Store<S>::ld(pop + slot) + shift : 0.0;
    }
  }
}

// resting fluid everywhere (f~ = 0) and the owner map of the face walls
template <class S>
__global__ void k_init(LatticeView lv) {
  const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= lv.N) return;
  S *pop = reinterpret_cast<S *>(lv.pop);
  for (int r = 0; r < Q; ++r) Store<S>::st(pop + (unsigned)r * lv.N + n, 0.0f);
  const int nx = lv.nx, ny = lv.ny, nz = lv.nz;
  const int c[3] = {(int)(n % nx), (int)((n / nx) % ny), (int)(n / ((unsigned)nx * ny))};
  const int dims[3] = {nx, ny, nz};
  int own = FLUID;
  for (int k = 0; k < 3 && own == FLUID; ++k) {
    if (lv.per[k]) continue;
    if (c[k] == 0) own = -2 - 2 * k;
    else if (c[k] == dims[k] - 1) own = -2 - (2 * k + 1);
  }
  lv.owner[n] = own;
}

__global__ void k_fill_int(int *a, unsigned n, int v) {
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

__global__ void k_apply_wall_mask(LatticeView lv, const uint8_t *mask) {
  const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= lv.N) return;
  if (mask[n]) lv.owner[n] = -2 - (int)(mask[n] - 1);
}

// ---------------------------------------------------------------------------
// surface wall nodes (walls with a non-wall neighbour, Sec. III) as bits

__global__ void k_surface_bits(LatticeView lv, SurfBits sb, int *count) {
  using D = D3Q19;
  const unsigned wi = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned nwords = (unsigned)sb.nxw * lv.ny * lv.nz;
  if (wi >= nwords) return;
  const int row = wi / sb.nxw, xw = wi % sb.nxw;
  const int y = row % lv.ny, z = row / lv.ny;
  uint32_t word = 0;
  for (int b = 0; b < 32; ++b) {
    const int x = 32 * xw + b;
    if (x >= lv.nx) break;
    const unsigned n = (unsigned)x + (unsigned)lv.nx * ((unsigned)y + (unsigned)lv.ny * z);
    if (lv.owner[n] > -2) continue;
    bool surf = false;
    for (int r = 1; r < Q && !surf; ++r) {
      const int xs = wrapi(x + D::cx(r), lv.nx), ys = wrapi(y + D::cy(r), lv.ny), zs = wrapi(z + D::cz(r), lv.nz);
      surf = lv.owner[(unsigned)xs + (unsigned)lv.nx * ((unsigned)ys + (unsigned)lv.ny * zs)] > -2;
    }
    if (surf) word |= 1u << b;
  }
  sb.bits[wi] = word;
  if (word) atomicAdd(count, __popc(word));
}

// ---------------------------------------------------------------------------
// link lists by warp-level stream compaction in node order:
// pass 0 counts per block, pass 1 writes at the block's scanned offset, each
// warp placing its lanes' links with ballot/popc prefix sums.

__global__ void k_links(LatticeView lv, int contact, int pass, int *block_count, const int *block_off, int32_t *out,
                        long long cap) {
  using D = D3Q19;
  __shared__ int warp_tot[32];
  __shared__ int warp_base[32];
  const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned mask = 0;
  int own = -2;
  if (n < lv.N) {
    own = lv.owner[n];
    const int nx = lv.nx, ny = lv.ny, nz = lv.nz;
    const int x = n % nx, y = (n / nx) % ny, z = n / ((unsigned)nx * ny);
    const bool src_ok = contact ? own >= 0 : own == FLUID;
    if (src_ok)
      for (int r = 1; r < Q; ++r) {
        const int xs = wrapi(x + D::cx(r), nx), ys = wrapi(y + D::cy(r), ny), zs = wrapi(z + D::cz(r), nz);
        const int on = lv.owner[(unsigned)xs + (unsigned)nx * ((unsigned)ys + (unsigned)ny * zs)];
        const bool hit = contact ? (on != FLUID && on != own) : (on != FLUID);
        if (hit) mask |= 1u << r;
      }
  }
  const int mine = __popc(mask);
  // inclusive scan of the lanes' counts
  int inc = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      warp_base[w] = s;
      s += warp_tot[w];
    }
    if (pass == 0) block_count[blockIdx.x] = s;
  }
  __syncthreads();
  if (pass == 0 || mine == 0) return;
  long long pos = (long long)block_off[blockIdx.x] + warp_base[wid] + (inc - mine);
  const int nx = lv.nx, ny = lv.ny, nz = lv.nz;
  const int x = n % nx, y = (n / nx) % ny, z = n / ((unsigned)nx * ny);
  for (int r = 1; r < Q; ++r) {
    if (!(mask & (1u << r))) continue;
    const int xs = wrapi(x + D::cx(r), nx), ys = wrapi(y + D::cy(r), ny), zs = wrapi(z + D::cz(r), nz);
    const int on = lv.owner[(unsigned)xs + (unsigned)nx * ((unsigned)ys + (unsigned)ny * zs)];
    if (pos < cap) {
      out[3 * pos + 0] = (int32_t)n;
      out[3 * pos + 1] = r;
      out[3 * pos + 2] = on;
    }
    ++pos;
  }
}

// ---------------------------------------------------------------------------
// host-side launchers

template <int PAR, bool FORCE, bool TAU1, int ZC>
static void launch_pipe(const LatticeView &lv, dim3 grid, dim3 block, const WallAcc &wa, int *status,
                        cudaStream_t st) {
  const dim3 gp(grid.x, grid.y, (grid.z + ZC - 1) / ZC);
  k_lb_step_pipe<PAR, FORCE, TAU1, ZC><<<gp, block, 0, st>>>(lv, wa, status);
}

template <class S, int PAR, bool FORCE, bool TAU1, int ZC, int TS>
static void launch_bulk(const LatticeView &lv, dim3 grid, const WallAcc &wa, int *status, cudaStream_t st) {
  const dim3 gp((lv.nx + 127) / 128, grid.y, (grid.z + ZC - 1) / ZC);
  k_lb_step_bulk<S, PAR, FORCE, TAU1, ZC, TS><<<gp, 128, 0, st>>>(lv, wa, status);
}

// row length for the bulk-copy sweep: 16-byte aligned rows of the storage type
__host__ __device__ inline bool bulk_rows_ok(int nx, int store_bytes) { return nx % (16 / store_bytes) == 0; }

// sweep variants (LatticeView::sweep): 0 one node per thread; 1, 2 the FP32
// pipeline over 4 or 8 planes; 3, 4 the bulk-copy pipeline over 8 or 4 planes
// with 3 stages (any storage type with 16-byte aligned rows, else variant 0)
template <class S, int PAR, bool FORCE, bool TAU1>
static void launch_lb_variant(const LatticeView &lv, dim3 grid, dim3 block, const WallAcc &wa, int *status,
                              cudaStream_t st) {
  if constexpr (std::is_same<S, float>::value) {
    if (lv.sweep == 1) return launch_pipe<PAR, FORCE, TAU1, 4>(lv, grid, block, wa, status, st);
    if (lv.sweep == 2) return launch_pipe<PAR, FORCE, TAU1, 8>(lv, grid, block, wa, status, st);
  }
  if (bulk_rows_ok(lv.nx, (int)sizeof(S))) {
    if (lv.sweep == 3) return launch_bulk<S, PAR, FORCE, TAU1, 8, 3>(lv, grid, wa, status, st);
    if (lv.sweep == 4) return launch_bulk<S, PAR, FORCE, TAU1, 4, 3>(lv, grid, wa, status, st);
  }
  k_lb_step<S, PAR, FORCE, TAU1><<<grid, block, 0, st>>>(lv, wa, status);
}

template <class S, int PAR, bool FORCE>
static void launch_lb_tau(const LatticeView &lv, dim3 grid, dim3 block, const WallAcc &wa, int *status,
                          cudaStream_t st) {
  if (lv.omega == 1.0f) launch_lb_variant<S, PAR, FORCE, true>(lv, grid, block, wa, status, st);
  else launch_lb_variant<S, PAR, FORCE, false>(lv, grid, block, wa, status, st);
}

template <class S>
static void launch_lb_typed(const LatticeView &lv, int par, const WallAcc &wa, int *status, cudaStream_t st) {
  const int bx = lv.nx >= 128 ? 128 : ((lv.nx + 31) / 32) * 32;
  dim3 block(bx, 1, 1);
  dim3 grid((lv.nx + bx - 1) / bx, lv.ny, lv.nz);
  if (par == 0) {
    if (lv.has_force) launch_lb_tau<S, 0, true>(lv, grid, block, wa, status, st);
    else launch_lb_tau<S, 0, false>(lv, grid, block, wa, status, st);
  } else {
    if (lv.has_force) launch_lb_tau<S, 1, true>(lv, grid, block, wa, status, st);
    else launch_lb_tau<S, 1, false>(lv, grid, block, wa, status, st);
  }
}

void launch_lb_step(int dtype, const LatticeView &lv, int par, const WallAcc &wa, int *status, cudaStream_t st) {
  if (dtype == 0) launch_lb_typed<float>(lv, par, wa, status, st);
  else if (dtype == 1) launch_lb_typed<__nv_bfloat16>(lv, par, wa, status, st);
  else launch_lb_typed<__half>(lv, par, wa, status, st);
}

static inline unsigned nblk(unsigned n, unsigned b) { return (n + b - 1) / b; }

void launch_geometry(const LatticeView &lv, const PartView &pv, cudaStream_t st, int64_t *nl) {
  const int bx = lv.nx >= 128 ? 128 : ((lv.nx + 31) / 32) * 32;
  dim3 grid((lv.nx + bx - 1) / bx, lv.ny, lv.nz);
  k_geometry<<<grid, bx, 0, st>>>(lv, pv);
  if (nl) ++*nl;
}

void launch_fields(int dtype, const LatticeView &lv, int par, double *rho, double *u, int32_t *owner, cudaStream_t st) {
  const unsigned b = 256, g = nblk(lv.N, b);
  if (dtype == 0) k_fields<float><<<g, b, 0, st>>>(lv, par, rho, u, owner);
  else if (dtype == 1) k_fields<__nv_bfloat16><<<g, b, 0, st>>>(lv, par, rho, u, owner);
  else k_fields<__half><<<g, b, 0, st>>>(lv, par, rho, u, owner);
}

void launch_pop_io(int dtype, const LatticeView &lv, int par, double *buf, int to_storage, cudaStream_t st) {
  const unsigned b = 256, g = nblk(lv.N, b);
  if (dtype == 0) k_pop_io<float><<<g, b, 0, st>>>(lv, par, buf, to_storage);
  else if (dtype == 1) k_pop_io<__nv_bfloat16><<<g, b, 0, st>>>(lv, par, buf, to_storage);
  else k_pop_io<__half><<<g, b, 0, st>>>(lv, par, buf, to_storage);
}

void launch_init(int dtype, const LatticeView &lv, cudaStream_t st) {
  const unsigned b = 256, g = nblk(lv.N, b);
  if (dtype == 0) k_init<float><<<g, b, 0, st>>>(lv);
  else if (dtype == 1) k_init<__nv_bfloat16><<<g, b, 0, st>>>(lv);
  else k_init<__half><<<g, b, 0, st>>>(lv);
}

void launch_fill_int(int *a, unsigned n, int v, cudaStream_t st) {
  k_fill_int<<<nblk(n, 256), 256, 0, st>>>(a, n, v);
}

void launch_apply_wall_mask(const LatticeView &lv, const uint8_t *mask, cudaStream_t st) {
  const unsigned b = 256, g = nblk(lv.N, b);
  k_apply_wall_mask<<<g, b, 0, st>>>(lv, mask);
}

void launch_surface_bits(const LatticeView &lv, const SurfBits &sb, int *count, cudaStream_t st) {
  const unsigned words = (unsigned)sb.nxw * lv.ny * lv.nz;
  k_surface_bits<<<nblk(words, 128), 128, 0, st>>>(lv, sb, count);
}

unsigned links_blocks(const LatticeView &lv) { return nblk(lv.N, 256); }

void launch_links(const LatticeView &lv, int contact, int pass, int *block_count, const int *block_off, int32_t *out,
                  long long cap, cudaStream_t st) {
  k_links<<<nblk(lv.N, 256), 256, 0, st>>>(lv, contact, pass, block_count, block_off, out, cap);
}

}  // namespace bl
