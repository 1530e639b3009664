// lb_kernels.cu -- the lattice sweep of the coupled step and the lattice-side
// helper kernels.
//
// The sweep fuses, per node and per time step (arXiv:1005.2594, Sec. II):
//   * moments rho, j and the Guo-forced velocity u = (j + rho g / 2) / rho,
//   * BGK collision (Eq. col) with the third-order equilibrium (Eq. neq),
//   * advection (Eq. adv) in the AA pattern on one buffer,
//   * mid-link bounce-back (Eq. lbe-bb) with the moving-boundary term C
//     (Eqs. c, lbe-bb-corr), evaluated at the link midpoint,
//   * the momentum exchange of each bounced link (Eq. deltap) into the force
//     and torque of the cell or the momentum counter of the wall,
//   * on cell nodes, the contact links to other cells and walls (Eqs.
//     deltapppp, deltapppm).
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
// Forces.  The momentum of a bounced link is (2 f*_r + C) c_r.  Its constant
// part 2 alpha_r rho_bar c_r = (rho_bar / 18) m_r c_r is accumulated exactly as
// integers (K, and IT for the torque, with the integer part of the lever
// arm); only the small variable part (2 f~*_r + C) c_r goes through floating
// point.  Lanes of a warp combine their sums per cell (match on the owner id,
// shuffle reduction) before one FP64 atomic per cell and component.
#include "bl_internal.cuh"

namespace bl {

namespace {

constexpr int KEY_NONE = 0x7fffffff;

struct Acc {
  int key;  // cell id >= 0, wall -2-w, or KEY_NONE
  float F[3], T[3];
  int K[3], I[3];
};

__device__ __forceinline__ void acc_clear(Acc &a) {
  a.key = KEY_NONE;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    a.F[k] = a.T[k] = 0.f;
    a.K[k] = a.I[k] = 0;
  }
}

__device__ __forceinline__ void acc_flush_direct(const Acc &a, const PartAcc &pa, const WallAcc &wa) {
  if (a.key == KEY_NONE) return;
  if (a.key >= 0) {
    const int p = a.key;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      atomicAdd(&pa.F[3 * p + k], (double)a.F[k]);
      atomicAdd(&pa.T[3 * p + k], (double)a.T[k]);
      atomicAdd(&pa.K[3 * p + k], a.K[k]);
      atomicAdd(&pa.IT[3 * p + k], a.I[k]);
    }
  } else {
    const int w = -2 - a.key;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      atomicAdd(&wa.F[3 * w + k], (double)a.F[k]);
      atomicAdd((unsigned long long *)&wa.K[3 * w + k], (unsigned long long)(long long)a.K[k]);
    }
  }
}

// switches the thread's accumulator to key, flushing a different one
__device__ __forceinline__ void acc_use(Acc &a, int key, const PartAcc &pa, const WallAcc &wa) {
  if (a.key == key) return;
  if (a.key != KEY_NONE) {
    acc_flush_direct(a, pa, wa);
    acc_clear(a);
  }
  a.key = key;
}

// warp-level combination: one atomic per distinct key of the warp
__device__ __forceinline__ void acc_warp_flush(Acc &a, const PartAcc &pa, const WallAcc &wa) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  unsigned pending = __ballot_sync(FULL, a.key != KEY_NONE);
  while (pending) {
    const int leader = __ffs(pending) - 1;
    const int lk = __shfl_sync(FULL, a.key, leader);
    const bool mine = a.key == lk;
    float v[6];
    int iv[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      v[k] = mine ? a.F[k] : 0.f;
      v[3 + k] = mine ? a.T[k] : 0.f;
      iv[k] = mine ? a.K[k] : 0;
      iv[3 + k] = mine ? a.I[k] : 0;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      v[k] = warp_sum(v[k]);
      iv[k] = __reduce_add_sync(FULL, iv[k]);
    }
    if (lane == leader) {
      if (lk >= 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          atomicAdd(&pa.F[3 * lk + k], (double)v[k]);
          atomicAdd(&pa.T[3 * lk + k], (double)v[3 + k]);
          atomicAdd(&pa.K[3 * lk + k], iv[k]);
          atomicAdd(&pa.IT[3 * lk + k], iv[3 + k]);
        }
      } else {
        const int w = -2 - lk;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          atomicAdd(&wa.F[3 * w + k], (double)v[k]);
          atomicAdd((unsigned long long *)&wa.K[3 * w + k], (unsigned long long)(long long)iv[k]);
        }
      }
    }
    pending &= ~__ballot_sync(FULL, mine);
    if (mine) a.key = KEY_NONE;
  }
}

}  // namespace

template <class S, int PAR>
__global__ void __launch_bounds__(128) k_lb_step(LatticeView lv, const float4 *__restrict__ kin, PartAcc pa,
                                                 WallAcc wa, LinkList ll, int *status) {
  using D = D3Q19;
  const int nx = lv.nx, ny = lv.ny;
  const int x0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  const bool valid = x0 < nx;
  const int x = valid ? x0 : nx - 1;
  const unsigned N = lv.N;
  const unsigned nxy = (unsigned)nx * (unsigned)ny;
  const unsigned n = (unsigned)x + (unsigned)nx * (unsigned)y + nxy * (unsigned)z;
  // coordinates of the 3 x 3 x 3 neighbourhood, periodic wrap on every axis
  // (a walled axis has wall layers at both ends, never crossed by a link)
  const unsigned xo[3] = {(unsigned)(x == 0 ? nx - 1 : x - 1), (unsigned)x, (unsigned)(x == nx - 1 ? 0 : x + 1)};
  const unsigned yo[3] = {(unsigned)(y == 0 ? ny - 1 : y - 1) * nx, (unsigned)y * nx,
                          (unsigned)(y == ny - 1 ? 0 : y + 1) * nx};
  const unsigned zo[3] = {(unsigned)(z == 0 ? lv.nz - 1 : z - 1) * nxy, (unsigned)z * nxy,
                          (unsigned)(z == lv.nz - 1 ? 0 : z + 1) * nxy};
  S *pop = reinterpret_cast<S *>(lv.pop);
  const int own = valid ? lv.owner[n] : -2;

  Acc acc;
  acc_clear(acc);
  unsigned part = 0;  // bit r: x + c_r is a cell node (a bounce link to record)
  float rho_node = 0.f;

  if (own == FLUID) {
    // owners of the 18 neighbours: bit r set when x + c_r is solid
    unsigned solid = 0;
    sfor<1, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      const unsigned nb = xo[1 + D::cx(r)] + yo[1 + D::cy(r)] + zo[1 + D::cz(r)];
      const int on = lv.owner[nb];
      solid |= (on != FLUID ? 1u : 0u) << r;
      part |= (on >= 0 ? 1u : 0u) << r;
    });
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
      f[r] = Store<S>::ld(pop + src);
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
    rho_node = rho;
    const float inv = 1.0f / rho;
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    if (lv.has_force) {
      Fx = rho * lv.g[0];
      Fy = rho * lv.g[1];
      Fz = rho * lv.g[2];
    }
    const float ux = (jx + 0.5f * Fx) * inv, uy = (jy + 0.5f * Fy) * inv, uz = (jz + 0.5f * Fz) * inv;
    const float uu = ux * ux + uy * uy + uz * uz;
    if (!(rho > 0.f) || !(uu < 0.09f)) atomicOr(status, ST_UNSTABLE);
    const float om = lv.omega;
    const float src_w = 1.0f - 0.5f * om;
    // collision in place: f[r] <- f~*_r
    sfor<0, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      constexpr float w = D::m(r) / 36.0f;
      const float cu = D::cx(r) * ux + D::cy(r) * uy + D::cz(r) * uz;
      const float t = cu * (3.0f + cu * (4.5f + 4.5f * cu)) - uu * (1.5f + 4.5f * cu);
      // rho t = rho_bar t + drho t keeps the small deviation exact in FP32
      const float feq = w * (drho + lv.rho0 * t + drho * t);
      float fs = f[r] - om * (f[r] - feq);
      if (lv.has_force) {
        const float cF = D::cx(r) * Fx + D::cy(r) * Fy + D::cz(r) * Fz;
        const float S = w * (3.0f * (cF - (ux * Fx + uy * Fy + uz * Fz)) + 9.0f * cu * cF);
        fs += src_w * S;
      }
      f[r] = fs;
    });
    Store<S>::st(pop + n, f[0]);
    sfor<1, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      constexpr int rb = D::opp(r);
      const unsigned nb = xo[1 + D::cx(r)] + yo[1 + D::cy(r)] + zo[1 + D::cz(r)];
      if (!(solid & (1u << r))) {
        const unsigned dst = PAR == 0 ? (unsigned)rb * N + n : (unsigned)r * N + nb;
        Store<S>::st(pop + dst, f[r]);
      } else {
        const unsigned dst = PAR == 0 ? (unsigned)r * N + nb : (unsigned)rb * N + n;
        const int on = lv.owner[nb];
        float vx, vy, vz;
        float ax = 0.f, ay = 0.f, az = 0.f;
        int dix = 0, diy = 0, diz = 0;
        if (on <= -2) {
          const int w = -2 - on;
          vx = lv.wall_vel[w][0];
          vy = lv.wall_vel[w][1];
          vz = lv.wall_vel[w][2];
        } else {
          const float4 k0 = __ldg(&kin[3 * on + 0]);
          const float4 k1 = __ldg(&kin[3 * on + 1]);
          const float4 k2 = __ldg(&kin[3 * on + 2]);
          dix = imin_image(x - (int)k0.w, nx, lv.per[0]);
          diy = imin_image(y - (int)k1.w, ny, lv.per[1]);
          diz = imin_image(z - (int)k2.w, lv.nz, lv.per[2]);
          // lever arm of the link midpoint x + c_r / 2 - X (Sec. II; reading Q2)
          ax = (float)dix + 0.5f * D::cx(r) - k0.x;
          ay = (float)diy + 0.5f * D::cy(r) - k0.y;
          az = (float)diz + 0.5f * D::cz(r) - k0.z;
          vx = k1.x + (k2.y * az - k2.z * ay);
          vy = k1.y + (k2.z * ax - k2.x * az);
          vz = k1.z + (k2.x * ay - k2.y * ax);
        }
        // C for the population returning along rbar: 6 alpha_rbar rho c_rbar . v
        const float C = -(D::m(r) / 6.0f) * rho * (D::cx(r) * vx + D::cy(r) * vy + D::cz(r) * vz);
        Store<S>::st(pop + dst, f[r] + C);
        // momentum to the solid: (2 f*_r + C) c_r, variable part here
        const float dp = 2.0f * f[r] + C;
        acc_use(acc, on, pa, wa);
        acc.F[0] += dp * D::cx(r);
        acc.F[1] += dp * D::cy(r);
        acc.F[2] += dp * D::cz(r);
        acc.K[0] += D::m(r) * D::cx(r);
        acc.K[1] += D::m(r) * D::cy(r);
        acc.K[2] += D::m(r) * D::cz(r);
        if (on >= 0) {
          const float px = dp * D::cx(r), py = dp * D::cy(r), pz = dp * D::cz(r);
          acc.T[0] += ay * pz - az * py;
          acc.T[1] += az * px - ax * pz;
          acc.T[2] += ax * py - ay * px;
          acc.I[0] += D::m(r) * (diy * D::cz(r) - diz * D::cy(r));
          acc.I[1] += D::m(r) * (diz * D::cx(r) - dix * D::cz(r));
          acc.I[2] += D::m(r) * (dix * D::cy(r) - diy * D::cx(r));
        }
      }
    });
  } else if (own >= 0) {
    // contact links of a cell node: -2 alpha_r rho_bar c_r per link to another
    // cell or a wall (Eqs. deltapppp, deltapppm), constant part only
    const float4 k0 = __ldg(&kin[3 * own + 0]);
    const float4 k1 = __ldg(&kin[3 * own + 1]);
    const float4 k2 = __ldg(&kin[3 * own + 2]);
    const int dix = imin_image(x - (int)k0.w, nx, lv.per[0]);
    const int diy = imin_image(y - (int)k1.w, ny, lv.per[1]);
    const int diz = imin_image(z - (int)k2.w, lv.nz, lv.per[2]);
    sfor<1, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      const unsigned nb = xo[1 + D::cx(r)] + yo[1 + D::cy(r)] + zo[1 + D::cz(r)];
      const int on = lv.owner[nb];
      if (on != FLUID && on != own) {
        acc.key = own;
        acc.K[0] -= D::m(r) * D::cx(r);
        acc.K[1] -= D::m(r) * D::cy(r);
        acc.K[2] -= D::m(r) * D::cz(r);
        acc.I[0] -= D::m(r) * (diy * D::cz(r) - diz * D::cy(r));
        acc.I[1] -= D::m(r) * (diz * D::cx(r) - dix * D::cz(r));
        acc.I[2] -= D::m(r) * (dix * D::cy(r) - diy * D::cx(r));
      }
    });
  }
  acc_warp_flush(acc, pa, wa);
  // warp-level compaction of this sweep's cell bounce links into the link list
  {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int mine = __popc(part);
    int inc = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += v;
    }
    const int tot = __shfl_sync(FULL, inc, 31);
    int base = 0;
    if (lane == 31 && tot) base = atomicAdd(ll.count, tot);
    base = __shfl_sync(FULL, base, 31);
    int pos = base + inc - mine;
    while (part) {
      const int r = __ffs(part) - 1;
      part &= part - 1;
      const unsigned nb = xo[1 + D::cx(r)] + yo[1 + D::cy(r)] + zo[1 + D::cz(r)];
      if (pos < ll.cap) {
        ll.node[pos] = n;
        ll.pr[pos] = ((unsigned)lv.owner[nb] << 5) | (unsigned)r;
        ll.rho[pos] = rho_node;
      } else {
        atomicOr(status, ST_OVERFLOW);
      }
      ++pos;
    }
  }
}

// ---------------------------------------------------------------------------
// implicit coupling over the recorded bounce links (reading Q3): the link
// force is linear in the cell velocity, F = F0 - Zff V - Zft W,
// T = T0 - Ztf V - Ztt W, with Z = sum (m_r / 6) rho [c; a x c][c; a x c]^T

__device__ __forceinline__ void link_geometry(const LatticeView &lv, const float4 *kin, uint32_t node, uint32_t pr,
                                              int &pid, int &r, float a[3], int xyz[3]) {
  using D = D3Q19;
  pid = (int)(pr >> 5);
  r = (int)(pr & 31u);
  const int nx = lv.nx, ny = lv.ny;
  xyz[0] = node % nx;
  xyz[1] = (node / nx) % ny;
  xyz[2] = node / ((unsigned)nx * ny);
  const float4 k0 = __ldg(&kin[3 * pid + 0]);
  const float4 k1 = __ldg(&kin[3 * pid + 1]);
  const float4 k2 = __ldg(&kin[3 * pid + 2]);
  a[0] = (float)imin_image(xyz[0] - (int)k0.w, nx, lv.per[0]) + 0.5f * D::cx(r) - k0.x;
  a[1] = (float)imin_image(xyz[1] - (int)k1.w, ny, lv.per[1]) + 0.5f * D::cy(r) - k0.y;
  a[2] = (float)imin_image(xyz[2] - (int)k2.w, lv.nz, lv.per[2]) + 0.5f * D::cz(r) - k0.z;
}

__global__ void __launch_bounds__(256) k_link_zeta(LatticeView lv, const float4 *__restrict__ kin, LinkList ll,
                                                   double *zeta) {
  using D = D3Q19;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int count = min(*ll.count, ll.cap);
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < count; base += stride) {
    const int i = base + threadIdx.x;
    int key = -1;
    float v[21];
#pragma unroll
    for (int k = 0; k < 21; ++k) v[k] = 0.f;
    if (i < count) {
      int pid, r, xyz[3];
      float a[3];
      link_geometry(lv, kin, ll.node[i], ll.pr[i], pid, r, a, xyz);
      const float c[3] = {(float)D::cx(r), (float)D::cy(r), (float)D::cz(r)};
      const float b[3] = {a[1] * c[2] - a[2] * c[1], a[2] * c[0] - a[0] * c[2], a[0] * c[1] - a[1] * c[0]};
      const float w = (D::m(r) / 6.0f) * ll.rho[i];
      int k = 0;
      for (int p = 0; p < 3; ++p)
        for (int q = p; q < 3; ++q) v[k++] = w * c[p] * c[q];
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) v[k++] = w * c[p] * b[q];
      for (int p = 0; p < 3; ++p)
        for (int q = p; q < 3; ++q) v[k++] = w * b[p] * b[q];
      key = pid;
    }
    unsigned pending = __ballot_sync(FULL, key >= 0);
    while (pending) {
      const int leader = __ffs(pending) - 1;
      const int lk = __shfl_sync(FULL, key, leader);
      const bool m = key == lk;
#pragma unroll
      for (int k = 0; k < 21; ++k) {
        const float s = warp_sum(m ? v[k] : 0.f);
        if (lane == leader) atomicAdd(&zeta[21 * lk + k], (double)s);
      }
      pending &= ~__ballot_sync(FULL, m);
      if (m) key = -1;
    }
  }
}

// adds C(new) - C(predictor) = -(m_r / 6) rho c_r . (dV + dW x a) to the
// population each recorded link bounced, in the layout of parity PAR
template <class S, int PAR>
__global__ void __launch_bounds__(256) k_link_correct(LatticeView lv, const float4 *__restrict__ kin, LinkList ll,
                                                      const float *__restrict__ dvel) {
  using D = D3Q19;
  const int count = min(*ll.count, ll.cap);
  S *pop = reinterpret_cast<S *>(lv.pop);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    int pid, r, xyz[3];
    float a[3];
    link_geometry(lv, kin, ll.node[i], ll.pr[i], pid, r, a, xyz);
    const float *d = dvel + 6 * pid;
    const float dvx = d[0] + (d[4] * a[2] - d[5] * a[1]);
    const float dvy = d[1] + (d[5] * a[0] - d[3] * a[2]);
    const float dvz = d[2] + (d[3] * a[1] - d[4] * a[0]);
    const float dC = -(D::m(r) / 6.0f) * ll.rho[i] * (D::cx(r) * dvx + D::cy(r) * dvy + D::cz(r) * dvz);
    const unsigned n = ll.node[i];
    unsigned dst;
    if (PAR == 0) {
      const int xs = wrapi(xyz[0] + D::cx(r), lv.nx), ys = wrapi(xyz[1] + D::cy(r), lv.ny),
                zs = wrapi(xyz[2] + D::cz(r), lv.nz);
      dst = (unsigned)r * lv.N + (unsigned)xs + (unsigned)lv.nx * ((unsigned)ys + (unsigned)lv.ny * zs);
    } else {
      dst = (unsigned)D::opp(r) * lv.N + n;
    }
    Store<S>::st(pop + dst, Store<S>::ld(pop + dst) + dC);
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
// surface wall nodes (walls with a non-wall neighbour, Sec. III), stored per
// lattice row (y, z) as sorted x coordinates

__global__ void k_surface_rows(LatticeView lv, int *row_count, int *row_x, const int *row_start) {
  using D = D3Q19;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= lv.ny * lv.nz) return;
  const int y = row % lv.ny, z = row / lv.ny;
  int cnt = 0;
  int out = row_start ? row_start[row] : 0;
  for (int x = 0; x < lv.nx; ++x) {
    const unsigned n = (unsigned)x + (unsigned)lv.nx * ((unsigned)y + (unsigned)lv.ny * z);
    if (lv.owner[n] > -2) continue;
    bool surf = false;
    for (int r = 1; r < Q && !surf; ++r) {
      const int xs = wrapi(x + D::cx(r), lv.nx), ys = wrapi(y + D::cy(r), lv.ny), zs = wrapi(z + D::cz(r), lv.nz);
      surf = lv.owner[(unsigned)xs + (unsigned)lv.nx * ((unsigned)ys + (unsigned)lv.ny * zs)] > -2;
    }
    if (!surf) continue;
    if (row_x) row_x[out++] = x;
    ++cnt;
  }
  if (row_count) row_count[row] = cnt;
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

template <class S>
static void launch_lb_typed(const LatticeView &lv, int par, const float4 *kin, const PartAcc &pa, const WallAcc &wa,
                            const LinkList &ll, int *status, cudaStream_t st) {
  const int bx = lv.nx >= 128 ? 128 : ((lv.nx + 31) / 32) * 32;
  dim3 block(bx, 1, 1);
  dim3 grid((lv.nx + bx - 1) / bx, lv.ny, lv.nz);
  if (par == 0)
    k_lb_step<S, 0><<<grid, block, 0, st>>>(lv, kin, pa, wa, ll, status);
  else
    k_lb_step<S, 1><<<grid, block, 0, st>>>(lv, kin, pa, wa, ll, status);
}

void launch_lb_step(int dtype, const LatticeView &lv, int par, const float4 *kin, const PartAcc &pa,
                    const WallAcc &wa, const LinkList &ll, int *status, cudaStream_t st) {
  if (dtype == 0) launch_lb_typed<float>(lv, par, kin, pa, wa, ll, status, st);
  else if (dtype == 1) launch_lb_typed<__nv_bfloat16>(lv, par, kin, pa, wa, ll, status, st);
  else launch_lb_typed<__half>(lv, par, kin, pa, wa, ll, status, st);
}

static unsigned link_grid() { return 152 * 8; }

void launch_link_zeta(const LatticeView &lv, const PartView &pv, const LinkList &ll, cudaStream_t st, int64_t *nl) {
  k_link_zeta<<<link_grid(), 256, 0, st>>>(lv, pv.kin, ll, pv.zeta);
  *nl += 1;
}

template <class S>
static void link_correct_typed(const LatticeView &lv, int par, const PartView &pv, const LinkList &ll,
                               cudaStream_t st) {
  if (par == 0) k_link_correct<S, 0><<<link_grid(), 256, 0, st>>>(lv, pv.kin, ll, pv.dvel);
  else k_link_correct<S, 1><<<link_grid(), 256, 0, st>>>(lv, pv.kin, ll, pv.dvel);
}

void launch_link_correct(int dtype, const LatticeView &lv, int par, const PartView &pv, const LinkList &ll,
                         cudaStream_t st, int64_t *nl) {
  if (dtype == 0) link_correct_typed<float>(lv, par, pv, ll, st);
  else if (dtype == 1) link_correct_typed<__nv_bfloat16>(lv, par, pv, ll, st);
  else link_correct_typed<__half>(lv, par, pv, ll, st);
  *nl += 1;
}

static inline unsigned nblk(unsigned n, unsigned b) { return (n + b - 1) / b; }

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

void launch_surface_rows(const LatticeView &lv, int *row_count, int *row_x, const int *row_start, cudaStream_t st) {
  const unsigned rows = (unsigned)lv.ny * lv.nz, b = 128;
  k_surface_rows<<<nblk(rows, b), b, 0, st>>>(lv, row_count, row_x, row_start);
}

unsigned links_blocks(const LatticeView &lv) { return nblk(lv.N, 256); }

void launch_links(const LatticeView &lv, int contact, int pass, int *block_count, const int *block_off, int32_t *out,
                  long long cap, cudaStream_t st) {
  k_links<<<nblk(lv.N, 256), 256, 0, st>>>(lv, contact, pass, block_count, block_off, out, cap);
}

}  // namespace bl
