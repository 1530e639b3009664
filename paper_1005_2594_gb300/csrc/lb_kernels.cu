// lb_kernels.cu -- the lattice-side helper kernels of the coupled step: the
// lattice-wide geometry pass, field and checkpoint read-outs, initial state,
// wall masks, surface wall nodes and link read-outs; and the dispatch of the
// lattice sweep (lb_sweep.cuh) to its storage types.
//
// Geometry pass.  After lb_init, walls_set and a first particles_set one
// lattice-wide pass (k_geometry) writes each fluid node's neighbour word --
// so the sweep reads one word per node instead of 18 neighbour owners --
// clears the pending moving-boundary terms and, at each cell node, sums its
// contact links.  Inside the steps the same results come incrementally
// (particle_kernels.cu: k_nbm_update, k_contacts).
#include "bl_internal.cuh"

namespace bl {

// ---------------------------------------------------------------------------
// geometry pass over the owner map (one thread per node, 128 along x)
//
//   fluid node  -> neighbour word (NB_* bits); no pending C (the pass runs
//                  where none is pending: after lb_init, walls_set, and a
//                  first particles_set, each of which gives pending C to the
//                  populations first)
//   cell node x of cell p, neighbour x + c_r another cell or a wall -> contact
//                  link (Eqs. deltapppp, deltapppm): its constant momentum
//                  -2 alpha_r rho_bar c_r goes into p's exact integer sums
//                  cK = sum m_r c_r, cIT = sum m_r dI x c_r, dI = x - rint(X_p)
//
// A warp adds its contact sums cell by cell with one atomic per value.  The
// sums start at zero (the claims kernel clears them).
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
  unsigned cmask = 0;
  if (valid) reinterpret_cast<float *>(lv.pu + n)[3] = 0.f;  // no pending C
  if (own >= FLUID) {
    unsigned solid = 0, wall = 0, same = 0;
    int first = -1;
    bool mixed = false;
    sfor<1, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      const unsigned nb = (unsigned)xs[1 + D::cx(r)] + (unsigned)nx * (unsigned)ys[1 + D::cy(r)] +
                          nxy * (unsigned)zs[1 + D::cz(r)];
      const int on = lv.owner[nb];
      solid |= (on != FLUID ? 1u : 0u) << r;
      wall |= (on <= -2 ? 1u : 0u) << r;
      same |= (on == own ? 1u : 0u) << r;
      if (on != FLUID) {
        if (first == -1) first = on;
        else if (on != first) mixed = true;
      }
    });
    if (own == FLUID) {
      lv.nbm[n] = NB_FLUID | solid | (wall ? NB_WALL : 0u) | ((solid & ~wall) ? NB_CELL : 0u);
      lv.nbc[n] = (first >= 0 && !mixed) ? (uint32_t)first : NBC_MIXED;
    } else {
      cmask = solid & ~same;  // other cells and walls
      lv.nbm[n] = cmask;
    }
  } else if (valid) {
    lv.nbm[n] = 0u;
  }
  if (pv.n == 0) return;  // no cell nodes: no contact links (uniform per launch)

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
  unsigned pend = __ballot_sync(FULL, cmask != 0u);
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

// the row bits: row (y, z) holds a surface wall node (rows cleared before)
__global__ void k_surface_rows(LatticeView lv, SurfBits sb) {
  const unsigned row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= (unsigned)lv.ny * lv.nz) return;
  uint32_t any = 0;
  for (int w = 0; w < sb.nxw; ++w) any |= sb.bits[(size_t)row * sb.nxw + w];
  if (any) atomicOr(&sb.rows[row >> 5], 1u << (row & 31));
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

// the sweep for each storage type (lb_sweep_f32.cu, lb_sweep_bf16.cu, lb_sweep_f16.cu)
void launch_lb_step_f32(const LatticeView &lv, int par, const WallAcc &wa, cudaStream_t st);
void launch_lb_step_bf16(const LatticeView &lv, int par, const WallAcc &wa, cudaStream_t st);
void launch_lb_step_f16(const LatticeView &lv, int par, const WallAcc &wa, cudaStream_t st);

void lb_rows_grids_f32(int out[8]);
void lb_rows_grids_bf16(int out[8]);
void lb_rows_grids_f16(int out[8]);

void lb_rows_grids(int dtype, int out[8]) {
  if (dtype == 0) lb_rows_grids_f32(out);
  else if (dtype == 1) lb_rows_grids_bf16(out);
  else lb_rows_grids_f16(out);
}

void launch_lb_step(int dtype, const LatticeView &lv0, int par, const WallAcc &wa, int *status, cudaStream_t st) {
  LatticeView lv = lv0;
  lv.status = status;
  if (dtype == 0) launch_lb_step_f32(lv, par, wa, st);
  else if (dtype == 1) launch_lb_step_bf16(lv, par, wa, st);
  else launch_lb_step_f16(lv, par, wa, st);
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

void launch_surface_rows(const LatticeView &lv, const SurfBits &sb, cudaStream_t st) {
  const unsigned rows = (unsigned)lv.ny * lv.nz;
  k_surface_rows<<<nblk(rows, 128), 128, 0, st>>>(lv, sb);
}

unsigned links_blocks(const LatticeView &lv) { return nblk(lv.N, 256); }

void launch_links(const LatticeView &lv, int contact, int pass, int *block_count, const int *block_off, int32_t *out,
                  long long cap, cudaStream_t st) {
  k_links<<<nblk(lv.N, 256), 256, 0, st>>>(lv, contact, pass, block_count, block_off, out, cap);
}


// ---------------------------------------------------------------------------
// Lees-Edwards shear (Sec. IV, reading Q25).  The images of the box along x
// slide past each other in z: the image above moves with velocity offset U
// and is displaced by D = U t (mod nz).  A population crossing the plane
// between x = nx - 1 and x = 0 therefore comes from the neighbouring image,
// from a point D along z from its periodic source -- between two nodes,
// interpolated linearly -- with its equilibrium part carried into this
// image's frame: n + n^eq(rho, u -+ U e_z) - n^eq(rho, u), with the moments of
// its source node.  Into x = 0 (c_x = +1) the source is
// (nx - 1, y - c_y, z - c_z + D) and the shift -U; into x = nx - 1 (c_x = -1)
// it is (0, y - c_y, z - c_z - D) and the shift +U.
//
// The sweep streams the crossing populations periodically; after each sweep
// two passes put the sheared values where the next read takes them.  After
// an even sweep (in place) population r of node s waits in slot rbar of s,
// and the odd sweep's node s + c_r reads it there; after an odd sweep it was
// written to slot r of s + c_r, where the even sweep reads it.  The gather
// forms each crossing population's shifted value from the moments the sweep
// left for its node (and the plane's momentum transfer); the scatter
// interpolates along z and writes the slots.  Both planes must hold fluid
// (ST_LEPLANE otherwise): the host allows no wall node, and cells are
// reflected before they reach them.

// the five directions with c_x = +1, and their opposites (c_x = -1)
__device__ constexpr int kLeUp[5] = {1, 7, 9, 11, 13};
__device__ constexpr int kLeDn[5] = {2, 8, 10, 12, 14};
static_assert(D3Q19::cx(1) == 1 && D3Q19::cx(7) == 1 && D3Q19::cx(9) == 1 && D3Q19::cx(11) == 1 &&
                  D3Q19::cx(13) == 1,
              "c_x = +1 directions");
static_assert(D3Q19::opp(1) == 2 && D3Q19::opp(7) == 8 && D3Q19::opp(9) == 10 && D3Q19::opp(11) == 12 &&
                  D3Q19::opp(13) == 14,
              "their opposites");

// t_r(u) of the third-order equilibrium n^eq_r = w_r rho (1 + t_r(u))
__device__ __forceinline__ float eq_t(float cu, float uu) {
  return cu * (3.0f + 4.5f * cu * cu - 4.5f * uu) + 4.5f * cu * cu - 1.5f * uu;
}

// node (x, y, z) + c_r, periodic
__device__ __forceinline__ unsigned le_node_plus(const LatticeView &lv, int x, int y, int z, int r) {
  using D = D3Q19;
  const int xx = x + D::cx(r), yy = y + D::cy(r), zz = z + D::cz(r);
  const int xw = xx < 0 ? xx + lv.nx : (xx >= lv.nx ? xx - lv.nx : xx);
  const int yw = yy < 0 ? yy + lv.ny : (yy >= lv.ny ? yy - lv.ny : yy);
  const int zw = zz < 0 ? zz + lv.nz : (zz >= lv.nz ? zz - lv.nz : zz);
  return (unsigned)xw + (unsigned)lv.nx * ((unsigned)yw + (unsigned)lv.ny * (unsigned)zw);
}

// one thread per node of the two planes: x = 0 (pl 0, its c_x = -1
// populations cross) and x = nx - 1 (pl 1, c_x = +1)
template <class S, int PAR>
__global__ void __launch_bounds__(128) k_le_gather(LatticeView lv, LeView le) {
  using D = D3Q19;
  const int ny = lv.ny, M = lv.ny * lv.nz;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const S *pop = reinterpret_cast<const S *>(lv.pop);
  float Pc = 0.f;
  if (i < 2 * M) {
    const int pl = i >= M ? 1 : 0;
    const int yz = i - pl * M, y = yz % ny, z = yz / ny;
    const int x = pl ? lv.nx - 1 : 0;
    const unsigned n = (unsigned)x + (unsigned)lv.nx * (unsigned)yz;
    if (!(lv.nbm[n] & NB_FLUID)) atomicOr(lv.status, ST_LEPLANE);
    const float4 m = lv.le_mom[i];
    const float rho = lv.rho0 + m.x;
    const float uz2 = m.w + (pl ? -(float)le.U : (float)le.U);
    const float uu = m.y * m.y + m.z * m.z + m.w * m.w, uu2 = m.y * m.y + m.z * m.z + uz2 * uz2;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const int r = pl ? kLeUp[k] : kLeDn[k];
      const float cx = (float)D::cx(r), cy = (float)D::cy(r), cz = (float)D::cz(r);
      const unsigned slot = PAR == 0 ? (unsigned)D::opp(r) * lv.N + n : (unsigned)r * lv.N + le_node_plus(lv, x, y, z, r);
      const float f = Store<S>::ld(pop + slot);
      const float cu = cx * m.y + cy * m.z + cz * m.w, cu2 = cx * m.y + cy * m.z + cz * uz2;
      const float dT = ((float)D::m(r) / 36.0f) * rho * (eq_t(cu2, uu2) - eq_t(cu, uu));
      le.T[(size_t)(pl * 5 + k) * M + yz] = f + dT;
      // z-momentum flux along +x through the plane, mean of the frame below
      // (c_x = +1 after the shift, c_x = -1 before) and above (the reverse)
      Pc += (pl ? 0.5f : -0.5f) * cz * (2.0f * f + dT);
    }
  }
  const float ws = warp_sum(Pc);
  if ((threadIdx.x & 31) == 0 && ws != 0.f) atomicAdd(le.P, (double)ws);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *le.D = fmod(le.U * (double)*le.t, (double)lv.nz);
    *le.t += 1;
    *le.n += 1;
  }
}

// one thread per node of the two planes: x = 0 (pl 0) receives the c_x = +1
// populations of x = nx - 1, x = nx - 1 (pl 1) the c_x = -1 ones of x = 0
template <class S, int PAR>
__global__ void __launch_bounds__(128) k_le_scatter(LatticeView lv, LeView le) {
  using D = D3Q19;
  const int ny = lv.ny, nz = lv.nz, M = lv.ny * lv.nz;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * M) return;
  S *pop = reinterpret_cast<S *>(lv.pop);
  const int pl = i >= M ? 1 : 0;
  const int yz = i - pl * M, y = yz % ny, z = yz / ny;
  const int x = pl ? lv.nx - 1 : 0;
  const unsigned n = (unsigned)x + (unsigned)lv.nx * (unsigned)yz;
  const double Dz = pl ? -*le.D : *le.D;
  const float *T = le.T + (size_t)(pl ? 0 : 5) * M;  // sources: x = 0 for pl 1, x = nx - 1 for pl 0
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int r = pl ? kLeDn[k] : kLeUp[k];
    const double zs = (double)(z - D::cz(r)) + Dz;
    const double z0 = floor(zs);
    const float w = (float)(zs - z0);
    int za = (int)z0 % nz;
    za = za < 0 ? za + nz : za;
    const int zb = za + 1 == nz ? 0 : za + 1;
    int ys = y - D::cy(r);
    ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
    const float a = T[(size_t)k * M + ys + ny * za], b = T[(size_t)k * M + ys + ny * zb];
    const float v = fmaf(w, b - a, a);
    // where the next sweep reads population r of node n
    const unsigned slot = PAR == 0 ? (unsigned)D::opp(r) * lv.N + le_node_plus(lv, x, y, z, D::opp(r))
                                   : (unsigned)r * lv.N + n;
    Store<S>::st(pop + slot, v);
  }
}

void launch_lees_edwards(int dtype, const LatticeView &lv, const LeView &le, int par, cudaStream_t st,
                         int64_t *nl) {
  const unsigned b = 128, g = nblk(2u * (unsigned)lv.ny * (unsigned)lv.nz, b);
#define BL_LE(S_)                                                   \
  if (par == 0) {                                                   \
    k_le_gather<S_, 0><<<g, b, 0, st>>>(lv, le);                    \
    k_le_scatter<S_, 0><<<g, b, 0, st>>>(lv, le);                   \
  } else {                                                          \
    k_le_gather<S_, 1><<<g, b, 0, st>>>(lv, le);                    \
    k_le_scatter<S_, 1><<<g, b, 0, st>>>(lv, le);                   \
  }
  if (dtype == 0) {
    BL_LE(float)
  } else if (dtype == 1) {
    BL_LE(__nv_bfloat16)
  } else {
    BL_LE(__half)
  }
#undef BL_LE
  if (nl) *nl += 2;
}

}  // namespace bl
