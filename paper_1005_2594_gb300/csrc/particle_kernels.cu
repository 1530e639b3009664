// particle_kernels.cu -- the cell side of the coupled step (arXiv:1005.2594):
//
//   cell list      count -> scan -> scatter -> per-bin sort, canonical (bin, id)
//   potentials     Berne-Pechukas-scaled Hookean cell-cell pairs (Sec. III,
//                  Eqs. phi, epsilon, sigma) and cell-wall spheres (Eq. sigmaw),
//                  one block per cell, FP64 contact geometry, FP32 forces,
//                  FP64 result
//   link sums      per cell over the link records the sweep wrote (Eq.
//                  deltap): link momentum at the predictor and the drag
//                  matrices
//   solve          one thread per cell: velocities of the half step (reading
//                  Q3), leap-frog on unit quaternions (reading Q4)
//   second links   the moving-boundary term C (Eq. c) on the rare links to a
//                  node's second cell; the first cell's C is added by the
//                  next sweep as it reads the bounced populations
//   claims         one block per cell, one thread per lattice row: the nodes
//                  the cell's new ellipsoid enters or leaves
//   resolve        first-arrival owner rule (Sec. II single occupancy), then
//                  fill/drain of every changed node with the momentum balance
//                  given to the cells (Sec. II)
//   contacts       contact links of each cell as exact integer sums (Eqs.
//                  deltapppp, deltapppm)
//
// Ownership.  claim[] holds INT_MAX ("free") on every node between steps.
// A cell marks each fluid node its new ellipsoid enters with its index
// (atomicMin: the lowest index among the newcomers) and each node it owns
// but leaves with TOUCHED; both go to the cell's touched list.  Resolve takes
// each claim once (atomicExch back to free): a newcomer index -> that cell;
// TOUCHED -> the lowest-index cell now covering the node, else fluid.  This
// is the first-arrival rule: an owner keeps a node while it covers it.
//
// FP64 is used only where the state needs it (positions, velocities, angular
// momenta, the exact inside test near a surface, the contact geometry of the
// potentials); on this GPU a one-lane FP64 instruction costs a full warp
// slot of a narrow pipe, so sums, the 6 x 6 solve and the rotation increment
// are FP32 around FP64 reference values.
#include <climits>

#include "bl_internal.cuh"

namespace bl {

constexpr int CLAIM_FREE = INT_MAX;
constexpr int CLAIM_TOUCHED = INT_MAX - 1;
// the FP32 inside test decides when |s - 1| >= this; its error is below
// 1e-5 for cells with half-axis ratios up to 100 (positions carried as an
// integer node plus an FP32 fraction)
constexpr float INSIDE_MARGIN = 1e-4f;

// ---------------------------------------------------------------------------
// cell list

__global__ void k_cl_bin(LatticeView lv, PartView pv, CellListView cl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pv.n) return;
  const int dims[3] = {lv.nx, lv.ny, lv.nz};
  int b[3];
  for (int k = 0; k < 3; ++k) {
    b[k] = (int)floor(__dmul_rn(__ddiv_rn(pv.X[3 * i + k], (double)dims[k]), (double)cl.nb[k]));
    if (b[k] < 0) b[k] = 0;
    if (b[k] > cl.nb[k] - 1) b[k] = cl.nb[k] - 1;
  }
  const int bin = b[0] + cl.nb[0] * (b[1] + cl.nb[1] * b[2]);
  cl.bin_of[i] = bin;
  atomicAdd(&cl.count[bin], 1);
}

// one block: exclusive scan of the bin counts into start, clears count/cursor
__global__ void __launch_bounds__(1024) k_cl_scan(CellListView cl) {
  __shared__ int wsum[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < cl.nbins; base += blockDim.x) {
    const int b = base + threadIdx.x;
    const int v = b < cl.nbins ? cl.count[b] : 0;
    int inc = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      int w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += t;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    const int excl = carry + (wid > 0 ? wsum[wid - 1] : 0) + inc - v;
    if (b < cl.nbins) {
      cl.start[b] = excl;
      cl.count[b] = 0;
      cl.cursor[b] = 0;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) cl.start[cl.nbins] = carry;
}

__global__ void k_cl_scatter(PartView pv, CellListView cl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pv.n) return;
  const int bin = cl.bin_of[i];
  const int slot = atomicAdd(&cl.cursor[bin], 1);
  cl.ids[cl.start[bin] + slot] = i;
}

__global__ void k_cl_sort(CellListView cl) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= cl.nbins) return;
  const int s = cl.start[b], e = cl.start[b + 1];
  for (int i = s + 1; i < e; ++i) {
    const int v = cl.ids[i];
    int j = i - 1;
    while (j >= s && cl.ids[j] > v) {
      cl.ids[j + 1] = cl.ids[j];
      --j;
    }
    cl.ids[j + 1] = v;
  }
}

// ---------------------------------------------------------------------------
// potentials (FP32)

// Contact geometry in FP64.  In contact the overlap h = 1 - r / sigma is a
// small difference of O(1) numbers (h ~ 1e-2), and the force is
// proportional to it: rounding r and sigma to FP32 (~1e-7) would put ~1e-5
// into the force.  So r (from the FP64 positions), the angles a, b, c, the
// shape function S, sigma and h are formed in FP64; the strength, its
// derivatives and the force and torque, which multiply h without cancelling
// it, in FP32.

// FP32 test of a pair against its contact distance (Eq. sigma) with a
// relative margin of 1e-4: false only for pairs certainly out of contact
__device__ __forceinline__ bool near_contact(const float r[3], float r2, const float oi[3], const float oj[3],
                                             const PartView &pv) {
  if (!(r2 > 0.f)) return false;
  const float ir = rsqrtf(r2);
  const float a = (r[0] * oi[0] + r[1] * oi[1] + r[2] * oi[2]) * ir;
  const float b = (r[0] * oj[0] + r[1] * oj[1] + r[2] * oj[2]) * ir;
  const float c = oi[0] * oj[0] + oi[1] * oj[1] + oi[2] * oj[2];
  const float chi = pv.chi, ap = a + b, am = a - b;
  const float S = 1.0f - 0.5f * chi * (ap * ap / (1.0f + chi * c) + am * am / (1.0f - chi * c));
  return r2 * S < pv.sigbar * pv.sigbar * 1.0002f;  // r < sigma_bar / sqrt(S) (1 + 1e-4)
}

// cell-cell pair, force and torque on i; r = X_j - X_i (Eqs. phi, epsilon,
// sigma; the Gay-Berne factor eps2^mu of the variant)
__device__ __forceinline__ void bp_pair(const double rd[3], const double oid[3], const double ojd[3],
                                        const PartView &pv, float F[3], float T[3]) {
  const double r2d = rd[0] * rd[0] + rd[1] * rd[1] + rd[2] * rd[2];
  if (!(r2d > 0.0)) return;
  const double rld = sqrt(r2d), ird = 1.0 / rld;
  const double rhd[3] = {rd[0] * ird, rd[1] * ird, rd[2] * ird};
  const double ad = rhd[0] * oid[0] + rhd[1] * oid[1] + rhd[2] * oid[2];
  const double bd = rhd[0] * ojd[0] + rhd[1] * ojd[1] + rhd[2] * ojd[2];
  const double cd = oid[0] * ojd[0] + oid[1] * ojd[1] + oid[2] * ojd[2];
  const double apd = ad + bd, amd = ad - bd;
  const double Sd = 1.0 - 0.5 * pv.chi_d * (apd * apd / (1.0 + pv.chi_d * cd) + amd * amd / (1.0 - pv.chi_d * cd));
  const double sigd = pv.sigbar_d / sqrt(Sd);
  if (rld >= sigd) return;
  const float h = (float)(1.0 - rld / sigd);
  const float rl = (float)rld, ir = (float)ird, sigma = (float)sigd, S = (float)Sd;
  const float rh[3] = {(float)rhd[0], (float)rhd[1], (float)rhd[2]};
  const float oi[3] = {(float)oid[0], (float)oid[1], (float)oid[2]};
  const float oj[3] = {(float)ojd[0], (float)ojd[1], (float)ojd[2]};
  const float a = (float)ad, b = (float)bd, c = (float)cd;
  const float chi = pv.chi;
  const float ap = (float)apd, am = (float)amd;
  const float dp = 1.0f + chi * c, dm = 1.0f - chi * c;
  const float e1 = 1.0f - chi * chi * c * c;
  float eps = pv.eps * (pv.nu == 1.0f ? rsqrtf(e1) : powf(e1, -0.5f * pv.nu));
  float e2 = 1.0f, de2a = 0.f, de2b = 0.f, de2c = 0.f;
  if (pv.mu != 0.0f) {
    const float cp = pv.chi_prime;
    const float qp = 1.0f + cp * c, qm = 1.0f - cp * c;
    e2 = 1.0f - 0.5f * cp * (ap * ap / qp + am * am / qm);
    de2a = -cp * (ap / qp + am / qm);
    de2b = -cp * (ap / qp - am / qm);
    de2c = 0.5f * cp * cp * (ap * ap / (qp * qp) - am * am / (qm * qm));
    eps *= powf(e2, pv.mu);
  }
  const float dSa = -chi * (ap / dp + am / dm);
  const float dSb = -chi * (ap / dp - am / dm);
  const float dSc = 0.5f * chi * chi * (ap * ap / (dp * dp) - am * am / (dm * dm));
  const float eps_a = pv.mu != 0.0f ? eps * pv.mu * de2a / e2 : 0.f;
  const float eps_b = pv.mu != 0.0f ? eps * pv.mu * de2b / e2 : 0.f;
  const float eps_c = eps * (pv.nu * chi * chi * c / e1 + (pv.mu != 0.0f ? pv.mu * de2c / e2 : 0.f));
  const float k = eps * h * rl / (sigma * S);
  const float phi_r = -2.0f * eps * h / sigma;
  const float phi_a = h * h * eps_a - k * dSa;
  const float phi_b = h * h * eps_b - k * dSb;
  const float phi_c = h * h * eps_c - k * dSc;
  float dpi[3];
  for (int m = 0; m < 3; ++m) {
    F[m] += phi_r * rh[m] + (phi_a * (oi[m] - a * rh[m]) + phi_b * (oj[m] - b * rh[m])) * ir;
    dpi[m] = phi_a * rh[m] + phi_c * oj[m];
  }
  T[0] -= oi[1] * dpi[2] - oi[2] * dpi[1];
  T[1] -= oi[2] * dpi[0] - oi[0] * dpi[2];
  T[2] -= oi[0] * dpi[1] - oi[1] * dpi[0];
}

// cell-wall sphere (Eq. sigmaw), force and torque on the cell; r = x_wall - X
__device__ __forceinline__ void bp_wall(const double rd[3], const double oid[3], const PartView &pv, float F[3],
                                        float T[3]) {
  const double r2d = rd[0] * rd[0] + rd[1] * rd[1] + rd[2] * rd[2];
  if (!(r2d > 0.0)) return;
  const double rld = sqrt(r2d), ird = 1.0 / rld;
  const double rhd[3] = {rd[0] * ird, rd[1] * ird, rd[2] * ird};
  const double ad = rhd[0] * oid[0] + rhd[1] * oid[1] + rhd[2] * oid[2];
  const double Dd = 1.0 - pv.chi_w_d * ad * ad;
  const double sigd = pv.sigbar_w_d / sqrt(Dd);
  if (rld >= sigd) return;
  const float h = (float)(1.0 - rld / sigd);
  const float rl = (float)rld, ir = (float)ird, sigma = (float)sigd, D = (float)Dd, a = (float)ad;
  const float rh[3] = {(float)rhd[0], (float)rhd[1], (float)rhd[2]};
  const float oi[3] = {(float)oid[0], (float)oid[1], (float)oid[2]};
  const float eps = pv.eps_w;
  const float dsig_a = sigma * pv.chi_w * a / D;
  const float phi_r = -2.0f * eps * h / sigma;
  const float phi_a = 2.0f * eps * h * rl / (sigma * sigma) * dsig_a;
  for (int m = 0; m < 3; ++m) F[m] += phi_r * rh[m] + phi_a * (oi[m] - a * rh[m]) * ir;
  const float dpo[3] = {phi_a * rh[0], phi_a * rh[1], phi_a * rh[2]};
  T[0] -= oi[1] * dpo[2] - oi[2] * dpo[1];
  T[1] -= oi[2] * dpo[0] - oi[0] * dpo[2];
  T[2] -= oi[0] * dpo[1] - oi[1] * dpo[0];
}

// neighbour-bin offsets along one axis without duplicates
__device__ __forceinline__ int bin_offsets(int nb, int per, int b, int out[3]) {
  if (nb == 1) {
    out[0] = 0;
    return 1;
  }
  if (nb == 2 && per) {
    out[0] = 0;
    out[1] = 1;
    return 2;
  }
  int k = 0;
  for (int d = -1; d <= 1; ++d) {
    const int v = b + d;
    if (!per && (v < 0 || v >= nb)) continue;
    out[k++] = d;
  }
  return k;
}

// ---------------------------------------------------------------------------
// block-wide helpers (blockDim.x == 256)

constexpr int CB = 256;

// sums v over a block of NT threads; the result is valid in thread 0
template <int K, int NT = CB>
__device__ __forceinline__ void block_sum(float (&v)[K], float (*sh)[K]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[wid][k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < NT / 32; ++w)
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] += sh[w][k];
  __syncthreads();
}

template <int K, int NT = CB>
__device__ __forceinline__ void block_sum_i(int (&v)[K], int (*sh)[K]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = __reduce_add_sync(0xffffffffu, v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[wid][k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < NT / 32; ++w)
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] += sh[w][k];
  __syncthreads();
}

// block-wide exclusive scan of one int per thread; returns the thread's
// offset, writes the total to *total (all threads)
template <int NT = CB>
__device__ __forceinline__ int block_scan(int v, int *sh_w, int *total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sh_w[wid] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < NT / 32; ++w) {
      const int t = sh_w[w];
      sh_w[w] = s;
      s += t;
    }
    sh_w[NT / 32] = s;
  }
  __syncthreads();
  const int off = sh_w[wid] + inc - v;
  *total = sh_w[NT / 32];
  __syncthreads();
  return off;
}

// per-warp append to a list whose length lives in shared memory: returns the
// first slot of this lane's cnt entries (one shared atomic per warp)
__device__ __forceinline__ int warp_append(int cnt, int *sh_len) {
  const int lane = threadIdx.x & 31;
  int inc = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  const int tot = __shfl_sync(0xffffffffu, inc, 31);
  int base = 0;
  if (lane == 31 && tot) base = atomicAdd(sh_len, tot);
  base = __shfl_sync(0xffffffffu, base, 31);
  return base + inc - cnt;
}

__device__ __forceinline__ unsigned node_of(const LatticeView &lv, int x, int y, int z) {
  return (unsigned)x + (unsigned)lv.nx * ((unsigned)y + (unsigned)lv.ny * z);
}

// walks the nodes of an inclusive box, CB threads at a time, without
// dividing per node: thread t starts at node t and advances by CB
struct BoxIter {
  int bx, by, bz, total;
  int ix, iy, iz, dx, dy, dz;
  __device__ void init(const int lo[3], const int hi[3]) {
    bx = hi[0] - lo[0] + 1;
    by = hi[1] - lo[1] + 1;
    bz = hi[2] - lo[2] + 1;
    total = (bx > 0 && by > 0 && bz > 0) ? bx * by * bz : 0;
    if (!total) return;
    const int t = threadIdx.x;
    iz = t / (bx * by);
    iy = (t / bx) % by;
    ix = t % bx;
    dz = CB / (bx * by);
    dy = (CB / bx) % by;
    dx = CB % bx;
  }
  __device__ void advance() {
    ix += dx;
    int c = 0;
    if (ix >= bx) {
      ix -= bx;
      c = 1;
    }
    iy += dy + c;
    c = 0;
    if (iy >= by) {
      iy -= by;
      c = 1;
    }
    iz += dz + c;
  }
};

// slot where the sweep of parity par bounced direction r of fluid node y
__device__ __forceinline__ unsigned bounce_slot(const LatticeView &lv, int par, unsigned y, const int yc[3], int r) {
  if (par == 0) {
    const unsigned nb = node_of(lv, wrapi(yc[0] + rt_c<0>(r), lv.nx), wrapi(yc[1] + rt_c<1>(r), lv.ny),
                                wrapi(yc[2] + rt_c<2>(r), lv.nz));
    return (unsigned)r * lv.N + nb;
  }
  return (unsigned)rt_opp(r) * lv.N + y;
}

// ---------------------------------------------------------------------------
// potentials: one block per cell.  Warp 0 takes the pairs (one lane per
// neighbouring bin), all threads take the rows (y, z) of the wall-sphere
// range around the cell.

constexpr int FB = 128;        // threads of a potentials block
constexpr int FQ_PAIR = 128;   // per-cell queue of pairs within contact reach
constexpr int FQ_WALL = 1024;  // per-cell queue of surface wall nodes within reach

// One block per cell.  The search runs in FP32 and queues what can be in
// contact: the cells j of the 27 bins around cell i within the largest
// contact distance (one thread per bin), and the surface wall nodes within
// the wall sphere's radius (rows without a surface wall node skipped by
// their row bit).  The queued pairs and wall nodes then get the FP64 contact
// geometry with one queue entry per thread, so that the few contacts of a
// cell share the FP64 instructions instead of each taking a pass of its own.
// A full queue evaluates the rest where they are found.
__global__ void __launch_bounds__(FB, 7) k_forces(LatticeView lv, PartView pv, CellListView cl, SurfBits sb) {
  __shared__ float sh[FB / 32][6];
  __shared__ int s_np, s_nw;
  __shared__ int s_pair[FQ_PAIR];
  __shared__ unsigned s_wall[FQ_WALL];
  const int i = blockIdx.x;
  if (threadIdx.x == 0) {
    s_np = 0;
    s_nw = 0;
  }
  __syncthreads();
  const float4 a0 = pv.kin[3 * i], a1 = pv.kin[3 * i + 1], a2 = pv.kin[3 * i + 2];
  const int Xi[3] = {(int)a0.w, (int)a1.w, (int)a2.w};
  const float fi[3] = {a0.x, a0.y, a0.z};
  // FP64 state of the step's start (the solve rewrites it only after the join)
  const double Xd[3] = {pv.X[3 * i], pv.X[3 * i + 1], pv.X[3 * i + 2]};
  const double oid[3] = {pv.o[3 * i], pv.o[3 * i + 1], pv.o[3 * i + 2]};
  const double fd[3] = {Xd[0] - (double)Xi[0], Xd[1] - (double)Xi[1], Xd[2] - (double)Xi[2]};  // exact
  const float oif[3] = {(float)oid[0], (float)oid[1], (float)oid[2]};
  const int dims[3] = {lv.nx, lv.ny, lv.nz};
  float F[3] = {0.f, 0.f, 0.f}, T[3] = {0.f, 0.f, 0.f};
  auto pair_force = [&](int j) {
    double rd[3];
    for (int m = 0; m < 3; ++m) rd[m] = min_image_exact(__dsub_rn(pv.X[3 * j + m], Xd[m]), dims[m], lv.per[m]);
    const double ojd[3] = {pv.o[3 * j], pv.o[3 * j + 1], pv.o[3 * j + 2]};
    bp_pair(rd, oid, ojd, pv, F, T);
  };
  // the wall node at offsets (dx, oy, oz) from rint(X); queued packed in
  // 3 x 10 bits (offsets within +-511, else evaluated where found)
  auto wall_force = [&](int dx, int oy, int oz) {
    const double rd[3] = {(double)dx - fd[0], (double)oy - fd[1], (double)oz - fd[2]};
    bp_wall(rd, oid, pv, F, T);
  };
  if (threadIdx.x < 27) {
    const int bin = cl.bin_of[i];
    const int bc[3] = {bin % cl.nb[0], (bin / cl.nb[0]) % cl.nb[1], bin / (cl.nb[0] * cl.nb[1])};
    int off[3][3], noff[3];
    for (int k = 0; k < 3; ++k) noff[k] = bin_offsets(cl.nb[k], lv.per[k], bc[k], off[k]);
    const int ix = threadIdx.x % 3, iy = (threadIdx.x / 3) % 3, iz = threadIdx.x / 9;
    if (ix < noff[0] && iy < noff[1] && iz < noff[2]) {
      const int bx = wrapi(bc[0] + off[0][ix], cl.nb[0]);
      const int by = wrapi(bc[1] + off[1][iy], cl.nb[1]);
      const int bz = wrapi(bc[2] + off[2][iz], cl.nb[2]);
      const int b = bx + cl.nb[0] * (by + cl.nb[1] * bz);
      const float rc2 = pv.r_cut * pv.r_cut;
      const float smax = 2.0f * fmaxf(pv.sig_par, pv.sig_perp);
      const float smax2 = smax * smax * 1.0001f;
      const int e = cl.start[b + 1];
      for (int k = cl.start[b]; k < e; ++k) {
        const int j = cl.ids[k];
        if (j == i) continue;
        const float4 b0 = pv.kin[3 * j], b1 = pv.kin[3 * j + 1], b2 = pv.kin[3 * j + 2];
        const int Xj[3] = {(int)b0.w, (int)b1.w, (int)b2.w};
        const float fj[3] = {b0.x, b0.y, b0.z};
        float r[3];
        for (int m = 0; m < 3; ++m) r[m] = (float)imin_image(Xj[m] - Xi[m], dims[m], lv.per[m]) + (fj[m] - fi[m]);
        const float r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        // no contact distance exceeds 2 max(sigma_perp, sigma_par); nearer
        // pairs first get the contact distance in FP32 (its error is ~1e-6
        // relative, far inside the margin): only pairs at or within contact
        // take the FP64 geometry
        if (r2 >= rc2 || r2 > smax2) continue;
        const float oj[3] = {(float)pv.o[3 * j], (float)pv.o[3 * j + 1], (float)pv.o[3 * j + 2]};
        if (!near_contact(r, r2, oif, oj, pv)) continue;
        const int q = atomicAdd(&s_np, 1);
        if (q < FQ_PAIR) s_pair[q] = j;
        else pair_force(j);
      }
    }
  }
  if (sb.bits) {
    const int R = (int)ceilf(pv.sigw_max) + 1;
    const int side = 2 * R + 1;
    const float rw2 = pv.sigw_max * pv.sigw_max;
    const bool packable = R <= 511;
    for (int t = threadIdx.x; t < side * side; t += FB) {
      const int oy = t % side - R, oz = t / side - R;  // node offsets from rint(X)
      int y = Xi[1] + oy, z = Xi[2] + oz;
      const float ry = (float)oy - fi[1], rz = (float)oz - fi[2];
      if (ry * ry + rz * rz >= rw2) continue;
      if (lv.per[1]) y = wrapi(y, lv.ny);
      else if (y < 0 || y >= lv.ny) continue;
      if (lv.per[2]) z = wrapi(z, lv.nz);
      else if (z < 0 || z >= lv.nz) continue;
      const unsigned ri = (unsigned)y + (unsigned)lv.ny * (unsigned)z;
      if (!((sb.rows[ri >> 5] >> (ri & 31)) & 1u)) continue;  // no surface wall node in the row
      const uint32_t *row = sb.bits + (size_t)ri * sb.nxw;
      for (int dx = -R; dx <= R; ++dx) {
        int x = Xi[0] + dx;
        if (lv.per[0]) x = wrapi(x, lv.nx);
        else if (x < 0 || x >= lv.nx) continue;
        if (!((row[x >> 5] >> (x & 31)) & 1u)) continue;
        // FP32 test against the wall sphere's radius first (margin 1e-4)
        const float rx = (float)dx - fi[0];
        const float r2 = rx * rx + ry * ry + rz * rz;
        const float af = rx * oif[0] + ry * oif[1] + rz * oif[2];
        if (!(r2 > 0.f) || (r2 - pv.chi_w * af * af) >= pv.sigbar_w * pv.sigbar_w * 1.0002f) continue;
        const int q = packable ? atomicAdd(&s_nw, 1) : FQ_WALL;
        if (q < FQ_WALL) s_wall[q] = (unsigned)(dx + 512) | ((unsigned)(oy + 512) << 10) | ((unsigned)(oz + 512) << 20);
        else wall_force(dx, oy, oz);
      }
    }
  }
  __syncthreads();
  // the queued contacts, one per thread
  const int np = min(s_np, FQ_PAIR), nw = min(s_nw, FQ_WALL);
  for (int k = threadIdx.x; k < np; k += FB) pair_force(s_pair[k]);
  for (int k = threadIdx.x; k < nw; k += FB) {
    const unsigned w = s_wall[k];
    wall_force((int)(w & 1023u) - 512, (int)((w >> 10) & 1023u) - 512, (int)(w >> 20) - 512);
  }
  float v[6] = {F[0], F[1], F[2], T[0], T[1], T[2]};
  block_sum<6, FB>(v, sh);
  if (threadIdx.x == 0)
    for (int m = 0; m < 3; ++m) {
      pv.Fpot[3 * i + m] = (double)v[m];
      pv.Tpot[3 * i + m] = (double)v[3 + m];
    }
}

// ---------------------------------------------------------------------------
// rigid-body helpers

__device__ void rotmat_f(const double q[4], float R[3][3]) {
  const float w = (float)q[0], x = (float)q[1], y = (float)q[2], z = (float)q[3];
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

// I_lab = R diag(I_perp, I_perp, I_par) R^T and its inverse (FP32)
__device__ void inertia_f(const PartView &pv, const double q[4], float I[3][3], float Iinv[3][3]) {
  float R[3][3];
  rotmat_f(q, R);
  const float d[3] = {(float)pv.Iperp, (float)pv.Iperp, (float)pv.Ipar};
  const float di[3] = {1.0f / d[0], 1.0f / d[1], 1.0f / d[2]};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      I[a][b] = R[a][0] * d[0] * R[b][0] + R[a][1] * d[1] * R[b][1] + R[a][2] * d[2] * R[b][2];
      Iinv[a][b] = R[a][0] * di[0] * R[b][0] + R[a][1] * di[1] * R[b][1] + R[a][2] * di[2] * R[b][2];
    }
}

// A x = b, A symmetric positive definite 6 x 6 (Cholesky, FP32)
__device__ void solve_spd6f(float A[6][6], const float b[6], float x[6]) {
  for (int j = 0; j < 6; ++j) {
    float d = A[j][j];
    for (int k = 0; k < j; ++k) d -= A[j][k] * A[j][k];
    d = sqrtf(d);
    A[j][j] = d;
    const float id = 1.0f / d;
    for (int i = j + 1; i < 6; ++i) {
      float v = A[i][j];
      for (int k = 0; k < j; ++k) v -= A[i][k] * A[j][k];
      A[i][j] = v * id;
    }
  }
  float y[6];
  for (int i = 0; i < 6; ++i) {
    float v = b[i];
    for (int k = 0; k < i; ++k) v -= A[i][k] * y[k];
    y[i] = v / A[i][i];
  }
  for (int i = 5; i >= 0; --i) {
    float v = y[i];
    for (int k = i + 1; k < 6; ++k) v -= A[k][i] * x[k];
    x[i] = v / A[i][i];
  }
}

__device__ void write_kin(const PartView &pv, int p, const double X[3], const double V[3], const double Om[3]) {
  double Xi[3], f[3];
  for (int k = 0; k < 3; ++k) {
    Xi[k] = rint(X[k]);
    f[k] = X[k] - Xi[k];
  }
  pv.kin_next[3 * p + 0] = make_float4((float)f[0], (float)f[1], (float)f[2], (float)Xi[0]);
  pv.kin_next[3 * p + 1] = make_float4((float)V[0], (float)V[1], (float)V[2], (float)Xi[1]);
  pv.kin_next[3 * p + 2] = make_float4((float)Om[0], (float)Om[1], (float)Om[2], (float)Xi[2]);
}

// X += V (wrapped), q <- exp(W / 2) (x) q with the rotation increment in FP32
// and a first-order renormalisation (|q|^2 - 1 is O(1e-7))
__device__ void rigid_advance(const LatticeView &lv, double X[3], double q[4], const double V[3], const double W[3]) {
  const int dims[3] = {lv.nx, lv.ny, lv.nz};
  for (int k = 0; k < 3; ++k) {
    X[k] += V[k];
    if (lv.per[k]) {
      if (X[k] < 0.0) X[k] += (double)dims[k];
      else if (X[k] >= (double)dims[k]) X[k] -= (double)dims[k];
    }
  }
  const float wx = (float)W[0], wy = (float)W[1], wz = (float)W[2];
  const float th = sqrtf(wx * wx + wy * wy + wz * wz);
  if (!(th > 0.f)) return;
  float sn, cs;
  sincosf(0.5f * th, &sn, &cs);
  const float sh = sn / th;
  const double dq[4] = {cs, wx * sh, wy * sh, wz * sh};
  double nq[4];
  nq[0] = dq[0] * q[0] - dq[1] * q[1] - dq[2] * q[2] - dq[3] * q[3];
  nq[1] = dq[0] * q[1] + dq[1] * q[0] + dq[2] * q[3] - dq[3] * q[2];
  nq[2] = dq[0] * q[2] - dq[1] * q[3] + dq[2] * q[0] + dq[3] * q[1];
  nq[3] = dq[0] * q[3] + dq[1] * q[2] - dq[2] * q[1] + dq[3] * q[0];
  const double nn = nq[0] * nq[0] + nq[1] * nq[1] + nq[2] * nq[2] + nq[3] * nq[3];
  const double c = 1.5 - 0.5 * nn;  // 1 / sqrt(nn) to second order in (nn - 1)
  for (int k = 0; k < 4; ++k) q[k] = nq[k] * c;
}

__device__ void aabb(const PartView &pv, const double X[3], const double o[3], int lo[3], int hi[3]) {
  for (int k = 0; k < 3; ++k) {
    const float ok = (float)o[k];
    const float h = sqrtf((float)(pv.R_perp * pv.R_perp) * (1.0f - ok * ok) + (float)(pv.R_par * pv.R_par) * ok * ok) + 0.01f;
    lo[k] = (int)floorf((float)X[k] - h);
    hi[k] = (int)ceilf((float)X[k] + h);
  }
}

// inside test: FP32 filter, exact FP64 re-evaluation near the surface
__device__ __forceinline__ bool inside_cell(int x, int y, int z, const double *X, const double *o, const float *Xf,
                                            const int *Xi, const float *of, const PartView &pv, const LatticeView &lv) {
  const float d0 = (float)imin_image(x - Xi[0], lv.nx, lv.per[0]) - Xf[0];
  const float d1 = (float)imin_image(y - Xi[1], lv.ny, lv.per[1]) - Xf[1];
  const float d2 = (float)imin_image(z - Xi[2], lv.nz, lv.per[2]) - Xf[2];
  const float dpar = d0 * of[0] + d1 * of[1] + d2 * of[2];
  const float dd = d0 * d0 + d1 * d1 + d2 * d2;
  const float s = dpar * dpar * (float)pv.inv_rpar2 + (dd - dpar * dpar) * (float)pv.inv_rperp2;
  if (fabsf(s - 1.0f) >= INSIDE_MARGIN) return s < 1.0f;
  return inside_exact(x, y, z, X, o, pv.inv_rpar2, pv.inv_rperp2, lv);
}

struct CellGeo {
  double X[3], o[3];
  float Xf[3], of[3];
  int Xi[3];
};

__device__ __forceinline__ void cell_geo(const PartView &pv, int p, CellGeo &g) {
  for (int k = 0; k < 3; ++k) {
    g.X[k] = pv.X[3 * p + k];
    g.o[k] = pv.o[3 * p + k];
    g.Xi[k] = (int)rint(g.X[k]);
    g.Xf[k] = (float)(g.X[k] - (double)g.Xi[k]);
    g.of[k] = (float)g.o[k];
  }
}

// ---------------------------------------------------------------------------
// implicit coupling (reading Q3).  The sweep bounced each cell's links
// without C and wrote one record per (fluid node, cell) into the cell's
// bucket.  With the predictor (Vp, Wp) = velocities of t-1/2 the link
// momentum is (2 f*_r + C(Vp, Wp)) c_r; the reduction sums it (variable part
// in FP32, 2 alpha_r rho_bar c_r as exact integers) with the drag matrices
// Z = sum (m_r / 6) rho [c; a x c][c; a x c]^T.  The half-step velocities
// V = Vp + dV, W = Wp + dW solve
//   (m + Zff) dV + Zft dW = F_tot(Vp, Wp) - m (Vp - V(t-1/2))
//   Ztf dV + (I + Ztt) dW = T_tot(Vp, Wp) + L(t-1/2) - I Wp,
// and the bounced populations get C(V, W) (the next sweep adds it as it
// reads them), so the fluid and the cell exchange the same momentum.
//
// All links of one node into a cell share d = y - X: the arm of link r is
// a_r = d + c_r / 2 and a_r x c_r = d x c_r.  So a record (rho, mask, F_raw =
// sum over the mask of 2 f~*_r c_r) gives
//   F0 = F_raw - rho M v_p,  T0 = d x F0,  v_p = Vp + Wp x d,
//   Zff = rho M,  Zft = rho M [d]x^T,  Ztt = [d]x rho M [d]x^T,
// with M = sum over the mask of (m_r / 6) c_r c_r^T, and the constant parts
// K = sum m_r c_r, IT = d_int x K with d_int = y - rint(X) exactly.  At
// tau = 1 the record holds the node's moments instead of F_raw, and the
// bounced populations f~*_r are evaluated again here by the function the
// sweep collides with.

constexpr int LT = 128;  // threads of a link-reduction block
// blocks of the link reduction and of the claims resident per SM: enough
// that one wave holds a thousand cells (the register cap this sets)
#ifndef BL_REDUCE_MINB
#define BL_REDUCE_MINB 7
#endif
#ifndef BL_CLAIMS_MINB
#define BL_CLAIMS_MINB 7
#endif
// threads of a block of the cell solve (one thread per cell): few, so that
// the FP64 work of the cells spreads over many SMs
#ifndef BL_SOLVE_TB
#define BL_SOLVE_TB 32
#endif

__global__ void __launch_bounds__(LT, BL_REDUCE_MINB) k_link_reduce(LatticeView lv, PartView pv) {
  __shared__ float shf[LT / 32][27];
  __shared__ int shi[LT / 32][6];
  __shared__ float4 cw[Q];  // (c_x, c_y, c_z, w_r) of each direction, for the masks' bits
  const int p = blockIdx.x;
  if (threadIdx.x < Q) {
    const int r = threadIdx.x;
    cw[r] = make_float4((float)D3::cx(r), (float)D3::cy(r), (float)D3::cz(r), (float)D3::m(r) / 36.0f);
  }
  __syncthreads();
  const int nrec = min(lv.rec_count[p], lv.rec_cap);
  const float4 k0 = pv.kin[3 * p], k1 = pv.kin[3 * p + 1], k2 = pv.kin[3 * p + 2];
  const int Xi[3] = {(int)k0.w, (int)k1.w, (int)k2.w};
  float v[27];
  int iv[6];
#pragma unroll
  for (int k = 0; k < 27; ++k) v[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 6; ++k) iv[k] = 0;
  const float4 *rec = lv.rec + 2 * (size_t)p * lv.rec_cap;
  const bool tau1 = lv.omega == 1.0f;  // the sweep's records hold moments (tau = 1) or link sums
  for (int i = threadIdx.x; i < nrec; i += LT) {
    const float4 r0 = rec[2 * i], r1 = rec[2 * i + 1];
    const unsigned n = __float_as_uint(r0.x);
    const uint32_t m = __float_as_uint(r0.y) & NB_SOLID;
    const float rho = lv.rho0 + r0.z;
    int yc[3];
    node_xyz(lv, n, yc);
    const int di[3] = {imin_image(yc[0] - Xi[0], lv.nx, lv.per[0]), imin_image(yc[1] - Xi[1], lv.ny, lv.per[1]),
                       imin_image(yc[2] - Xi[2], lv.nz, lv.per[2])};
    const float d[3] = {(float)di[0] - k0.x, (float)di[1] - k0.y, (float)di[2] - k0.z};
    // rho M and K from the mask
    const float w6 = rho * (1.0f / 6.0f);
    const float Axx = w6 * (float)mask_Maa<0>(m), Ayy = w6 * (float)mask_Maa<1>(m), Azz = w6 * (float)mask_Maa<2>(m);
    const float Axy = w6 * (float)mask_Mab<0, 1>(m), Axz = w6 * (float)mask_Mab<0, 2>(m),
                Ayz = w6 * (float)mask_Mab<1, 2>(m);
    const int K[3] = {mask_K<0>(m), mask_K<1>(m), mask_K<2>(m)};
    // the sum of 2 f~*_r c_r over the mask: at tau = 1 the bounced populations
    // again from the node's moments (drho, u, uu, uF), else the sweep's sums
    float Fr[3];
    if (tau1) {
      const float ux = r0.w, uy = r1.x, uz = r1.y, uu = r1.z, uF = r1.w;
      const float Fx = lv.has_force ? rho * lv.g[0] : 0.f, Fy = lv.has_force ? rho * lv.g[1] : 0.f,
                  Fz = lv.has_force ? rho * lv.g[2] : 0.f;
      Fr[0] = Fr[1] = Fr[2] = 0.f;
      for (uint32_t mm = m; mm; mm &= mm - 1u) {
        const float4 c = cw[__ffs(mm) - 1];
        const float cu = c.x * ux + c.y * uy + c.z * uz;
        const float cF = c.x * Fx + c.y * Fy + c.z * Fz;
        const float fs2 = 2.0f * post_tau1(c.w, r0.z, lv.rho0, cu, uu, lv.has_force != 0, cF, uF, 0.5f);
        Fr[0] += c.x * fs2;
        Fr[1] += c.y * fs2;
        Fr[2] += c.z * fs2;
      }
    } else {
      Fr[0] = r0.w;
      Fr[1] = r1.x;
      Fr[2] = r1.y;
    }
    const float A[3][3] = {{Axx, Axy, Axz}, {Axy, Ayy, Ayz}, {Axz, Ayz, Azz}};
    // predictor velocity at the node and the link momentum
    const float vp[3] = {k1.x + (k2.y * d[2] - k2.z * d[1]), k1.y + (k2.z * d[0] - k2.x * d[2]),
                         k1.z + (k2.x * d[1] - k2.y * d[0])};
    float F[3];
    F[0] = Fr[0] - (A[0][0] * vp[0] + A[0][1] * vp[1] + A[0][2] * vp[2]);
    F[1] = Fr[1] - (A[1][0] * vp[0] + A[1][1] * vp[1] + A[1][2] * vp[2]);
    F[2] = Fr[2] - (A[2][0] * vp[0] + A[2][1] * vp[1] + A[2][2] * vp[2]);
    v[0] += F[0];
    v[1] += F[1];
    v[2] += F[2];
    v[3] += d[1] * F[2] - d[2] * F[1];
    v[4] += d[2] * F[0] - d[0] * F[2];
    v[5] += d[0] * F[1] - d[1] * F[0];
    v[6] += Axx;
    v[7] += Axy;
    v[8] += Axz;
    v[9] += Ayy;
    v[10] += Ayz;
    v[11] += Azz;
    // G = A [d]x^T (the Zft block), then Ztt = [d]x G
    float G[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      G[a][0] = A[a][2] * d[1] - A[a][1] * d[2];
      G[a][1] = A[a][0] * d[2] - A[a][2] * d[0];
      G[a][2] = A[a][1] * d[0] - A[a][0] * d[1];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) v[12 + 3 * a + b] += G[a][b];
    v[21] += G[2][0] * d[1] - G[1][0] * d[2];
    v[22] += G[2][1] * d[1] - G[1][1] * d[2];
    v[23] += G[2][2] * d[1] - G[1][2] * d[2];
    v[24] += G[0][1] * d[2] - G[2][1] * d[0];
    v[25] += G[0][2] * d[2] - G[2][2] * d[0];
    v[26] += G[1][2] * d[0] - G[0][2] * d[1];
    iv[0] += K[0];
    iv[1] += K[1];
    iv[2] += K[2];
    iv[3] += di[1] * K[2] - di[2] * K[1];
    iv[4] += di[2] * K[0] - di[0] * K[2];
    iv[5] += di[0] * K[1] - di[1] * K[0];
  }
  // warp sums, then one thread per value adds the warps (FP64) and writes
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 27; ++k) {
    const float t = warp_sum(v[k]);
    if (lane == 0) shf[wid][k] = t;
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int t = __reduce_add_sync(0xffffffffu, iv[k]);
    if (lane == 0) shi[wid][k] = t;
  }
  __syncthreads();
  if (threadIdx.x < 27) {
    double t = 0.0;
    for (int w2 = 0; w2 < LT / 32; ++w2) t += (double)shf[w2][threadIdx.x];
    pv.lsum[27 * p + threadIdx.x] = t;
  } else if (threadIdx.x >= 32 && threadIdx.x < 38) {
    int t = 0;
    for (int w2 = 0; w2 < LT / 32; ++w2) t += shi[w2][threadIdx.x - 32];
    pv.lsum_i[6 * p + threadIdx.x - 32] = t;
  } else if (threadIdx.x == 64) {
    // the bucket is read: keep its size for the link read-out, empty it for the next sweep
    pv.rec_last[p] = nrec;
    lv.rec_count[p] = 0;
  }
}

// one thread per cell: link force at the predictor, 6 x 6 solve, leap-frog,
// kinematics and claim box of the next step
__global__ void k_solve(LatticeView lv, PartView pv) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= pv.n) return;
  const float4 k1 = pv.kin[3 * p + 1], k2 = pv.kin[3 * p + 2];
  double X[3], q[4], V[3], L[3], W[3], Xold[3], o_old[3];
  for (int k = 0; k < 3; ++k) {
    X[k] = pv.X[3 * p + k];
    V[k] = pv.V[3 * p + k];
    L[k] = pv.L[3 * p + k];
    W[k] = pv.Om[3 * p + k];
    Xold[k] = X[k];
    o_old[k] = pv.o[3 * p + k];
  }
  for (int k = 0; k < 4; ++k) q[k] = pv.q[4 * p + k];
  for (int k = 0; k < 3; ++k) pv.oprev[3 * p + k] = (float)o_old[k];  // the claims' old ellipsoid
  double vd[6];
  float v[27];
  for (int k = 0; k < 27; ++k) {
    v[k] = (float)pv.lsum[27 * p + k];
    if (k < 6) vd[k] = pv.lsum[27 * p + k];
  }
  double K[3], IT[3];
  for (int k = 0; k < 3; ++k) {
    // (the link reduction and the contact kernel rewrite these every step)
    K[k] = (double)(pv.lsum_i[6 * p + k] + pv.cK[3 * p + k]);
    IT[k] = (double)(pv.lsum_i[6 * p + 3 + k] + pv.cIT[3 * p + k]);
  }
  // link force at the predictor: variable part + exact constant part, with
  // f = X - rint(X) the fraction the sweep's lever arms used
  const double cst = pv.rho0 / 18.0;
  double f[3];
  for (int k = 0; k < 3; ++k) f[k] = X[k] - rint(X[k]);
  const double fxK[3] = {f[1] * K[2] - f[2] * K[1], f[2] * K[0] - f[0] * K[2], f[0] * K[1] - f[1] * K[0]};
  double Fl[3], Tl[3], Ft[3], Tt[3];
  for (int k = 0; k < 3; ++k) {
    Fl[k] = vd[k] + cst * K[k];
    Tl[k] = vd[3 + k] + cst * (IT[k] - fxK[k]);
    Ft[k] = Fl[k] + pv.Fpot[3 * p + k] + pv.PF[3 * p + k] + (pv.bfc ? pv.m * pv.g[k] : 0.0);
    Tt[k] = Tl[k] + pv.Tpot[3 * p + k] + pv.PT[3 * p + k];
    pv.PF[3 * p + k] = 0.0;
    pv.PT[3 * p + k] = 0.0;
  }
  const double Vp[3] = {k1.x, k1.y, k1.z}, Wp[3] = {k2.x, k2.y, k2.z};
  const bool move = pv.move != 0;
  if (pv.move == 1) {  // free cells; 2: prescribed, V and W stay as set
    float Z[6][6];
    {
      int k = 6;
      for (int s = 0; s < 3; ++s)
        for (int t = s; t < 3; ++t, ++k) Z[s][t] = Z[t][s] = v[k];
      for (int s = 0; s < 3; ++s)
        for (int t = 0; t < 3; ++t, ++k) Z[s][3 + t] = Z[3 + t][s] = v[k];
      for (int s = 0; s < 3; ++s)
        for (int t = s; t < 3; ++t, ++k) Z[3 + s][3 + t] = Z[3 + t][3 + s] = v[k];
    }
    float I[3][3], Iinv[3][3], A[6][6], rhs[6], d[6];
    inertia_f(pv, q, I, Iinv);
    for (int s = 0; s < 6; ++s)
      for (int t = 0; t < 6; ++t) A[s][t] = Z[s][t];
    for (int s = 0; s < 3; ++s) {
      A[s][s] += (float)pv.m;
      for (int t = 0; t < 3; ++t) A[3 + s][3 + t] += I[s][t];
      // L(t-1/2) - I Wp: a small difference of O(I W) numbers, in FP64
      const double IW = (double)I[s][0] * Wp[0] + (double)I[s][1] * Wp[1] + (double)I[s][2] * Wp[2];
      rhs[s] = (float)(Ft[s] - pv.m * (Vp[s] - V[s]));
      rhs[3 + s] = (float)(Tt[s] + (L[s] - IW));
    }
    solve_spd6f(A, rhs, d);
    for (int s = 0; s < 3; ++s) {
      float dF = 0.f, dT = 0.f;
      for (int t = 0; t < 6; ++t) {
        dF += Z[s][t] * d[t];
        dT += Z[3 + s][t] * d[t];
      }
      Fl[s] -= dF;
      Tl[s] -= dT;
      Ft[s] -= dF;
      Tt[s] -= dT;
    }
    for (int s = 0; s < 3; ++s) {
      V[s] = Vp[s] + (double)d[s];
      W[s] = Wp[s] + (double)d[3 + s];
      L[s] += Tt[s];
    }
  }
  for (int s = 0; s < 3; ++s) {
    pv.Flink[3 * p + s] = Fl[s];
    pv.Tlink[3 * p + s] = Tl[s];
    pv.Ftot[3 * p + s] = Ft[s];
    pv.Ttot[3 * p + s] = Tt[s];
    pv.vw[6 * p + s] = (float)V[s];
    pv.vw[6 * p + 3 + s] = (float)W[s];
  }
  int lo[3] = {0, 0, 0}, hi[3] = {-1, -1, -1};
  if (move) {
    // Sec. IV: a free cell closer than le_dr to the sheared plane (x = -1/2)
    // and moving toward it has its normal velocity negated; the step's
    // coupling above used the solve's velocity, the cell moves with the
    // reflected one (reading Q25)
    if (pv.le_dr > 0.0 && pv.move == 1) {
      const double dlo = X[0] + 0.5, dhi = (double)lv.nx - 0.5 - X[0];
      if ((dlo < pv.le_dr && V[0] < 0.0) || (dhi < pv.le_dr && V[0] > 0.0)) V[0] = -V[0];
    }
    rigid_advance(lv, X, q, V, W);
    for (int k = 0; k < 3; ++k) {
      pv.X[3 * p + k] = X[k];
      pv.V[3 * p + k] = V[k];
      pv.L[3 * p + k] = L[k];
      pv.Om[3 * p + k] = W[k];
    }
    for (int k = 0; k < 4; ++k) pv.q[4 * p + k] = q[k];
    double o_new[3];
    axis_exact(q, o_new);
    for (int k = 0; k < 3; ++k) pv.o[3 * p + k] = o_new[k];
    bool finite = true;
    for (int k = 0; k < 3; ++k) finite = finite && isfinite(X[k]) && isfinite(o_new[k]);
    // a cell faster than half a node per step is far outside the method's
    // low-Mach range (and would outrun the cell list of the step's start)
    if (!(V[0] * V[0] + V[1] * V[1] + V[2] * V[2] < 0.25)) finite = false;
    if (finite) {
      int lo2[3], hi2[3];
      aabb(pv, X, o_new, lo, hi);
      aabb(pv, Xold, o_old, lo2, hi2);
      const int dims[3] = {lv.nx, lv.ny, lv.nz};
      for (int k = 0; k < 3; ++k) {
        lo[k] = min(lo[k], lo2[k]);
        hi[k] = max(hi[k], hi2[k]);
        if (!lv.per[k]) {
          lo[k] = max(lo[k], 0);
          hi[k] = min(hi[k], dims[k] - 1);
        } else if (hi[k] - lo[k] + 1 > dims[k]) {
          lo[k] = 0;
          hi[k] = dims[k] - 1;
        }
      }
    } else {
      atomicOr(pv.status, ST_UNSTABLE);
    }
  }
  if (move)  // fixed cells keep the box of their last set: the geometry pass still needs it
    for (int k = 0; k < 3; ++k) {
      pv.box[6 * p + k] = lo[k];
      pv.box[6 * p + 3 + k] = hi[k];
    }
  write_kin(pv, p, X, V, W);
}

// The pending moving-boundary term of each record, right after the solve
// (one block per cell, beside the claims).  A record of a node's first cell
// becomes the node's pending velocity pu = rho (V + W x d) with its bounced
// directions, which the next sweep adds as C = -(m_r / 6) c_r . pu to the
// populations it reads; the records of a second or third cell of one node
// (marked REC_DIRECT) get their C in place.  V, W: the cell's half-step
// velocities of the solve; d: node minus the cell's position of this step.
// Every link is one cell's, so no two blocks touch the same slot.
template <class S>
__global__ void __launch_bounds__(LT) k_link_pending(LatticeView lv, PartView pv, int par) {
  constexpr int PQ = 512;  // queue of a block's second- and third-cell records
  __shared__ int s_nq;
  __shared__ int s_q[PQ];
  const int p = blockIdx.x;
  if (threadIdx.x == 0) s_nq = 0;
  __syncthreads();
  const int nrec = min(pv.rec_last[p], lv.rec_cap);
  const float4 k0 = pv.kin[3 * p], k1 = pv.kin[3 * p + 1], k2 = pv.kin[3 * p + 2];
  const int Xi[3] = {(int)k0.w, (int)k1.w, (int)k2.w};
  const float *vw = pv.vw + 6 * p;
  const float V[3] = {vw[0], vw[1], vw[2]}, W[3] = {vw[3], vw[4], vw[5]};
  S *pop = reinterpret_cast<S *>(lv.pop);
  const float4 *rec = lv.rec + 2 * (size_t)p * lv.rec_cap;
  // rho (V + W x d) of record i's node, its coordinates and its mask word
  auto node_u = [&](int i, unsigned &n, uint32_t &mb, int yc[3], float u[3]) {
    const float4 r0 = rec[2 * i];
    n = __float_as_uint(r0.x);
    mb = __float_as_uint(r0.y);
    node_xyz(lv, n, yc);
    const float d[3] = {(float)imin_image(yc[0] - Xi[0], lv.nx, lv.per[0]) - k0.x,
                        (float)imin_image(yc[1] - Xi[1], lv.ny, lv.per[1]) - k0.y,
                        (float)imin_image(yc[2] - Xi[2], lv.nz, lv.per[2]) - k0.z};
    const float rho = lv.rho0 + r0.z;
    u[0] = rho * (V[0] + (W[1] * d[2] - W[2] * d[1]));
    u[1] = rho * (V[1] + (W[2] * d[0] - W[0] * d[2]));
    u[2] = rho * (V[2] + (W[0] * d[1] - W[1] * d[0]));
  };
  // C in place for the directions of a second- or third-cell record
  auto direct = [&](int i) {
    unsigned n;
    uint32_t mb;
    int yc[3];
    float u[3];
    node_u(i, n, mb, yc, u);
    for (uint32_t m = mb & NB_SOLID; m; m &= m - 1u) {
      const int r = __ffs(m) - 1;
      const float C = -((float)rt_m(r) / 6.0f) * ((float)rt_c<0>(r) * u[0] + (float)rt_c<1>(r) * u[1] +
                                                  (float)rt_c<2>(r) * u[2]);
      const unsigned slot = bounce_slot(lv, par, n, yc, r);
      Store<S>::st(pop + slot, Store<S>::ld(pop + slot) + C);
    }
  };
  for (int i = threadIdx.x; i < nrec; i += LT) {
    const uint32_t mb = __float_as_uint(rec[2 * i].y);
    if (mb & REC_DIRECT) {
      const int k = atomicAdd(&s_nq, 1);
      if (k < PQ) s_q[k] = i;
      else direct(i);
      continue;
    }
    unsigned n;
    uint32_t mb2;
    int yc[3];
    float u[3];
    node_u(i, n, mb2, yc, u);
    lv.pu[n] = make_float4(u[0], u[1], u[2], __uint_as_float(mb2 & NB_SOLID));
  }
  // the records of a node's second or third cell, gathered so that the
  // warps take their per-direction loops with full lanes
  __syncthreads();
  const int nq = min(s_nq, PQ);
  for (int k = threadIdx.x; k < nq; k += LT) direct(s_q[k]);
}

// The pending C of the last step given to the stored populations, for
// read-outs and state changes between steps (the sweep's arithmetic); par is
// the layout of the stored populations (the next step's parity).
template <class S>
__global__ void k_flush_pending(LatticeView lv, int par) {
  using D = D3Q19;
  S *pop = reinterpret_cast<S *>(lv.pop);
  for (unsigned n = blockIdx.x * blockDim.x + threadIdx.x; n < lv.N; n += gridDim.x * blockDim.x) {
    const float4 pu = lv.pu[n];
    const uint32_t pm = __float_as_uint(pu.w);
    if (!pm) continue;
    int yc[3];
    node_xyz(lv, n, yc);
    for (uint32_t m = pm; m; m &= m - 1u) {
      const int r = __ffs(m) - 1;
      const float C = -(D::m(r) / 6.0f) * (D::cx(r) * pu.x + D::cy(r) * pu.y + D::cz(r) * pu.z);
      // the slot from which node n reads direction rbar in layout par
      const unsigned slot = bounce_slot(lv, par ^ 1, n, yc, r);
      Store<S>::st(pop + slot, Store<S>::ld(pop + slot) + C);
    }
    reinterpret_cast<float *>(lv.pu + n)[3] = 0.f;
  }
}

// particles_set: the state comes from the stage.  mode 1: first set (the
// box holds the new ellipsoid); mode 2: later set (old and new ellipsoid)
__global__ void k_set_state(LatticeView lv, PartView pv, int mode) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= pv.n) return;
  double Xold[3], o_old[3];
  for (int k = 0; k < 3; ++k) {
    Xold[k] = pv.X[3 * p + k];
    o_old[k] = pv.o[3 * p + k];
  }
  const double *st = pv.stage + 13 * p;
  double X[3], q[4], V[3], L[3], W[3];
  for (int k = 0; k < 3; ++k) {
    X[k] = st[k];
    V[k] = st[7 + k];
    L[k] = st[10 + k];
  }
  for (int k = 0; k < 4; ++k) q[k] = st[3 + k];
  float I[3][3], Iinv[3][3];
  inertia_f(pv, q, I, Iinv);
  for (int k = 0; k < 3; ++k)
    W[k] = (double)(Iinv[k][0] * (float)L[0] + Iinv[k][1] * (float)L[1] + Iinv[k][2] * (float)L[2]);
  for (int k = 0; k < 3; ++k) {
    pv.X[3 * p + k] = X[k];
    pv.V[3 * p + k] = V[k];
    pv.L[3 * p + k] = L[k];
    pv.Om[3 * p + k] = W[k];
    pv.vw[6 * p + k] = (float)V[k];
    pv.vw[6 * p + 3 + k] = (float)W[k];
  }
  for (int k = 0; k < 4; ++k) pv.q[4 * p + k] = q[k];
  double o_new[3];
  axis_exact(q, o_new);
  for (int k = 0; k < 3; ++k) {
    pv.oprev[3 * p + k] = (float)(mode == 2 ? o_old[k] : o_new[k]);
    pv.o[3 * p + k] = o_new[k];
  }
  write_kin(pv, p, X, V, W);
  int lo[3], hi[3], lo2[3], hi2[3];
  aabb(pv, X, o_new, lo, hi);
  bool finite = isfinite(X[0]) && isfinite(X[1]) && isfinite(X[2]);
  if (mode == 2) {
    finite = finite && isfinite(Xold[0]) && isfinite(Xold[1]) && isfinite(Xold[2]);
    aabb(pv, Xold, o_old, lo2, hi2);
    for (int k = 0; k < 3; ++k) {
      lo[k] = min(lo[k], lo2[k]);
      hi[k] = max(hi[k], hi2[k]);
    }
  }
  const int dims[3] = {lv.nx, lv.ny, lv.nz};
  for (int k = 0; k < 3; ++k) {
    if (!finite) {
      lo[k] = 0;
      hi[k] = -1;
    } else if (!lv.per[k]) {
      lo[k] = max(lo[k], 0);
      hi[k] = min(hi[k], dims[k] - 1);
    } else if (hi[k] - lo[k] + 1 > dims[k]) {
      lo[k] = 0;
      hi[k] = dims[k] - 1;
    }
    pv.box[6 * p + k] = lo[k];
    pv.box[6 * p + 3 + k] = hi[k];
  }
  if (!finite) atomicOr(pv.status, ST_UNSTABLE);
}

// Row intervals of an ellipsoid.  Along the lattice row (y, z) the inside
// function is a quadratic in t = x - X_x:
//   s(t) = A t^2 + B t + C0,  A = ip + kk o_x^2,  B = 2 kk o_x e,
//   C0 = (dy^2 + dz^2) ip + kk e^2,  e = o_y dy + o_z dz,
// ip = 1 / R_perp^2, kk = 1 / R_par^2 - 1 / R_perp^2 (A > 0 for any axis).
struct RowQuad {
  float A, B, C0;
};

__device__ __forceinline__ RowQuad row_quad(float dy, float dz, const float o[3], float ip, float kk) {
  const float e = o[1] * dy + o[2] * dz;
  return RowQuad{ip + kk * o[0] * o[0], 2.0f * kk * o[0] * e, (dy * dy + dz * dz) * ip + kk * e * e};
}

// node offsets i = x - rint(X_x) of the row with s <= L, as [lo, hi] (empty:
// lo > hi); xf = X_x - rint(X_x)
__device__ __forceinline__ void row_range(const RowQuad &q, float L, float xf, int &lo, int &hi) {
  const float disc = q.B * q.B - 4.0f * q.A * (q.C0 - L);
  if (!(disc >= 0.0f)) {
    lo = 1;
    hi = 0;
    return;
  }
  const float sq = sqrtf(disc), h = 0.5f / q.A;
  lo = (int)ceilf((-q.B - sq) * h + xf);
  hi = (int)floorf((-q.B + sq) * h + xf);
}

// Margin in s between the FP32 row intervals and the exact inside test: the
// FP32 interval ends are off by less than 1e-4 in s for half-axis ratios up
// to 100, so nodes with s <= 1 - ROW_EPS on a row's FP32 estimate are inside
// and nodes with s > 1 + ROW_EPS are outside.
constexpr float ROW_EPS = 2e-3f;

constexpr int PB = 128;  // threads of the claims and resolve blocks (8 blocks fit an SM)

// Claims (one block per cell, one thread per lattice row of the cell's box).
// A node's cover by cell p can change only where the old and the new
// ellipsoid differ: on each row, the nodes of the hull of the two outer
// intervals (s <= 1 + ROW_EPS) that are not in both inner ones (s <= 1 -
// ROW_EPS).  Those candidates get the exact inside test:
//   owned by p and no longer inside -> TOUCHED (resolve finds the new owner)
//   fluid and now inside            -> claim with p (atomicMin: lowest newcomer)
// Every node inside some cell is owned by a cell after each resolve, so a
// fluid node inside p is one that p's ellipsoid has just entered, and nodes
// owned by another cell need no claim: their owner keeps them while it
// covers them (first arrival), and hands them on through TOUCHED.
// mode 1: no old ellipsoid (first particles_set, all owners fluid).
// In particles_set (modes 1, 2) also clears the cell's link count and
// contact sums for the lattice-wide geometry pass, which adds to them; in a
// step (mode 0) the contact sums of this step are in use, and the next
// step's contact kernel rewrites them.
__global__ void __launch_bounds__(PB, BL_CLAIMS_MINB) k_claims(LatticeView lv, PartView pv, int *claim, ChangeList chg, int mode) {
  __shared__ int sh_len;
  const int p = blockIdx.x;
  if (threadIdx.x == 0) {
    sh_len = 0;
    if (mode != 0) {
      for (int k = 0; k < 3; ++k) {
        pv.cK[3 * p + k] = 0;
        pv.cIT[3 * p + k] = 0;
      }
    }
    if (p == 0) *chg.count = 0;
  }
  __syncthreads();
  const int lo1 = pv.box[6 * p + 1], lo2 = pv.box[6 * p + 2];
  const int by = pv.box[6 * p + 4] - lo1 + 1, bz = pv.box[6 * p + 5] - lo2 + 1;
  const int rows = (by > 0 && bz > 0) ? by * bz : 0;
  CellGeo g;
  cell_geo(pv, p, g);
  const bool has_old = mode != 1;
  int Xo[3] = {0, 0, 0};
  float xfo[3] = {0.f, 0.f, 0.f}, oo[3] = {0.f, 0.f, 0.f};
  if (has_old) {
    const float4 k0 = pv.kin[3 * p], k1 = pv.kin[3 * p + 1], k2 = pv.kin[3 * p + 2];
    Xo[0] = (int)k0.w;
    Xo[1] = (int)k1.w;
    Xo[2] = (int)k2.w;
    xfo[0] = k0.x;
    xfo[1] = k0.y;
    xfo[2] = k0.z;
    for (int k = 0; k < 3; ++k) oo[k] = pv.oprev[3 * p + k];
  }
  const float ip = (float)pv.inv_rperp2, kk = (float)(pv.inv_rpar2 - pv.inv_rperp2);
  const int shift = imin_image(Xo[0] - g.Xi[0], lv.nx, lv.per[0]);  // old rint(X_x) from the new one
  // offsets of one period (periodic x) or of the lattice (walled x)
  const int imin = lv.per[0] ? -(lv.nx / 2) : -g.Xi[0];
  const int imax = lv.per[0] ? imin + lv.nx - 1 : lv.nx - 1 - g.Xi[0];
  unsigned long long *touched = pv.touched + (size_t)p * pv.touched_cap;
  for (int t = threadIdx.x; t < rows; t += PB) {
    int y = lo1 + t % by, z = lo2 + t / by;
    if (lv.per[1]) y = wrapi(y, lv.ny);
    if (lv.per[2]) z = wrapi(z, lv.nz);
    const RowQuad qn = row_quad((float)imin_image(y - g.Xi[1], lv.ny, lv.per[1]) - g.Xf[1],
                                (float)imin_image(z - g.Xi[2], lv.nz, lv.per[2]) - g.Xf[2], g.of, ip, kk);
    int ao, bo, ai, bi;
    row_range(qn, 1.0f + ROW_EPS, g.Xf[0], ao, bo);
    row_range(qn, 1.0f - ROW_EPS, g.Xf[0], ai, bi);
    if (has_old) {
      const RowQuad qo = row_quad((float)imin_image(y - Xo[1], lv.ny, lv.per[1]) - xfo[1],
                                  (float)imin_image(z - Xo[2], lv.nz, lv.per[2]) - xfo[2], oo, ip, kk);
      int ao2, bo2, ai2, bi2;
      row_range(qo, 1.0f + ROW_EPS, xfo[0], ao2, bo2);
      row_range(qo, 1.0f - ROW_EPS, xfo[0], ai2, bi2);
      if (ao2 <= bo2) {
        if (ao > bo) {
          ao = ao2 + shift;
          bo = bo2 + shift;
        } else {
          ao = min(ao, ao2 + shift);
          bo = max(bo, bo2 + shift);
        }
      }
      if (ai2 <= bi2) {
        ai = max(ai, ai2 + shift);
        bi = min(bi, bi2 + shift);
      } else {
        ai = 1;
        bi = 0;
      }
    } else {
      ai = 1;  // nothing was covered: every node of the new interval
      bi = 0;
    }
    ao = max(ao, imin);
    bo = min(bo, imax);
    if (ao > bo) continue;
    // candidates: [ao, bo] without the common core [ai, bi]
    const bool core = ai <= bi;
    const int e1 = core ? min(bo, ai - 1) : bo;
    const int s2 = core ? max(ao, bi + 1) : bo + 1;
    for (int i = ao; i <= bo; ++i) {
      if (i > e1 && i < s2) {
        i = s2 - 1;
        continue;
      }
      int x = g.Xi[0] + i;
      if (lv.per[0]) x = wrapi(x, lv.nx);
      const unsigned idx = node_of(lv, x, y, z);
      const int ow = lv.owner[idx];
      int mark = 0;
      if (ow == p) {
        if (!inside_cell(x, y, z, g.X, g.o, g.Xf, g.Xi, g.of, pv, lv)) {
          atomicMin(&claim[idx], CLAIM_TOUCHED);
          mark = 1;
        }
      } else if (ow == FLUID) {
        if (inside_cell(x, y, z, g.X, g.o, g.Xf, g.Xi, g.of, pv, lv)) {
          atomicMin(&claim[idx], p);
          mark = 1;
        }
      }
      if (mark) {
        const int pos = atomicAdd(&sh_len, 1);
        if (pos < pv.touched_cap) touched[pos] = pack_xyzr(x, y, z, 0);
        else atomicOr(pv.status, ST_OVERFLOW);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) pv.touched_count[p] = min(sh_len, pv.touched_cap);
}

// lowest-index cell whose ellipsoid covers node (x, y, z), FLUID if none.
// Cells are searched in the node's bin and its neighbours: a bin is at least
// r_cut wide, r_cut exceeds the largest half-axis by one node, and a cell
// moves less than half a node per step, so the cell list of the step's start
// holds every cover of the node.  Bins list their cells in index order.
// (one warp per node: lane b < 27 scans neighbouring bin b, the lowest
// covering index over the lanes wins; all 32 lanes call it)
__device__ int lowest_cover(const LatticeView &lv, const PartView &pv, const CellListView &cl, int x, int y,
                                 int z) {
  const int lane = threadIdx.x & 31;
  const int c[3] = {x, y, z};
  const int dims[3] = {lv.nx, lv.ny, lv.nz};
  int bc[3], off[3][3], noff[3];
  for (int k = 0; k < 3; ++k) {
    bc[k] = (int)(((long long)c[k] * cl.nb[k]) / dims[k]);
    noff[k] = bin_offsets(cl.nb[k], lv.per[k], bc[k], off[k]);
  }
  int best = INT_MAX;
  const int ix = lane % 3, iy = (lane / 3) % 3, iz = lane / 9;
  if (lane < 27 && ix < noff[0] && iy < noff[1] && iz < noff[2]) {
    const int b = wrapi(bc[0] + off[0][ix], cl.nb[0]) +
                  cl.nb[0] * (wrapi(bc[1] + off[1][iy], cl.nb[1]) + cl.nb[1] * wrapi(bc[2] + off[2][iz], cl.nb[2]));
    const int e = cl.start[b + 1];
    for (int k = cl.start[b]; k < e; ++k) {
      const int j = cl.ids[k];
      CellGeo g;
      cell_geo(pv, j, g);
      if (inside_cell(x, y, z, g.X, g.o, g.Xf, g.Xi, g.of, pv, lv)) {
        best = j;
        break;
      }
    }
  }
  best = __reduce_min_sync(0xffffffffu, best);
  return best == INT_MAX ? FLUID : best;
}

// ---------------------------------------------------------------------------
// resolve + fill/drain over each cell's touched nodes

__device__ __forceinline__ void atomic_add3(double *a, const double v[3]) {
  atomicAdd(a, v[0]);
  atomicAdd(a + 1, v[1]);
  atomicAdd(a + 2, v[2]);
}

template <class S>
__global__ void __launch_bounds__(PB) k_resolve_fill(LatticeView lv, PartView pv, CellListView cl, int *claim,
                                                      ChangeList chg, int par_next, int impulses) {
  using D = D3Q19;
  const int p = blockIdx.x;
  const unsigned long long *touched = pv.touched + (size_t)p * pv.touched_cap;
  // the first touched node of this thread is requested with the count (the
  // list holds touched_cap entries)
  unsigned long long tv0 = 0ull;
  if ((int)threadIdx.x < pv.touched_cap) tv0 = touched[threadIdx.x];
  const int nt = pv.touched_count[p];
  const int lane = threadIdx.x & 31;
  S *pop = reinterpret_cast<S *>(lv.pop);
  const int dims[3] = {lv.nx, lv.ny, lv.nz};
  __shared__ int s_need[PB], s_res[PB];
  __shared__ int s_ns;
  for (int t0 = 0; t0 < nt; t0 += PB) {
    const int t = t0 + threadIdx.x;
    int old = 0, nw = 0, xyz[3] = {0, 0, 0};
    bool changed = false, act = false, need = false;
    unsigned idx = 0;
    if (threadIdx.x == 0) s_ns = 0;
    __syncthreads();
    if (t < nt) {
      int r_unused;
      unpack_xyzr(t0 == 0 ? tv0 : touched[t], xyz, r_unused);
      idx = node_of(lv, xyz[0], xyz[1], xyz[2]);
      const int own = lv.owner[idx];  // requested beside the claim's exchange
      const int c = atomicExch(&claim[idx], CLAIM_FREE);
      if (c != CLAIM_FREE) {
        act = true;
        old = own;
        // TOUCHED: the old owner left the node -> the lowest-index cell now
        // covering it (searched below by a warp), else fluid; a claim: a
        // fluid node entered by the claimants, the lowest of which takes it
        // (reading Q5)
        if (c == CLAIM_TOUCHED) {
          need = true;
          s_need[atomicAdd(&s_ns, 1)] = threadIdx.x;
        } else {
          nw = c;
        }
      }
    }
    __syncthreads();
    for (int k = threadIdx.x >> 5; k < s_ns; k += PB / 32) {
      const int tt = s_need[k];
      int cc[3], r_unused;
      unpack_xyzr(touched[t0 + tt], cc, r_unused);
      const int best = lowest_cover(lv, pv, cl, cc[0], cc[1], cc[2]);
      if (lane == 0) s_res[tt] = best;
    }
    __syncthreads();
    if (act) {
      if (need) nw = s_res[threadIdx.x];
      changed = nw != old;
      if (changed) lv.owner[idx] = nw;
    }
    // warp-level compaction of the changed nodes into the diagnostic list
    const unsigned bal = __ballot_sync(0xffffffffu, changed);
    int wbase = 0;
    if (lane == 0 && bal) wbase = atomicAdd(chg.count, __popc(bal));
    wbase = __shfl_sync(0xffffffffu, wbase, 0);
    if (!changed) continue;
    const int pos = wbase + __popc(bal & ((1u << lane) - 1u));
    if (pos < chg.cap) {
      chg.items[3 * pos] = (int32_t)idx;
      chg.items[3 * pos + 1] = old;
      chg.items[3 * pos + 2] = nw;
    }
    unsigned slot[Q];
    for (int r = 0; r < Q; ++r) {
      if (par_next == 0 || r == 0) {
        slot[r] = (unsigned)r * lv.N + idx;
      } else {
        slot[r] = (unsigned)D::opp(r) * lv.N +
                  node_of(lv, wrapi(xyz[0] - D::cx(r), lv.nx), wrapi(xyz[1] - D::cy(r), lv.ny),
                          wrapi(xyz[2] - D::cz(r), lv.nz));
      }
    }
    double arm_o[3] = {0, 0, 0}, arm_n[3] = {0, 0, 0};
    float u_o[3] = {0.f, 0.f, 0.f};
    if (old >= 0) {
      for (int k = 0; k < 3; ++k) arm_o[k] = min_image_exact((double)xyz[k] - pv.X[3 * old + k], dims[k], lv.per[k]);
      const double *W = pv.Om + 3 * old;
      u_o[0] = (float)(pv.V[3 * old + 0] + (W[1] * arm_o[2] - W[2] * arm_o[1]));
      u_o[1] = (float)(pv.V[3 * old + 1] + (W[2] * arm_o[0] - W[0] * arm_o[2]));
      u_o[2] = (float)(pv.V[3 * old + 2] + (W[0] * arm_o[1] - W[1] * arm_o[0]));
    }
    if (nw >= 0)
      for (int k = 0; k < 3; ++k) arm_n[k] = min_image_exact((double)xyz[k] - pv.X[3 * nw + k], dims[k], lv.per[k]);
    if (old == FLUID && nw >= 0) {
      // covered: the fluid is deleted, its momentum goes to the new owner;
      // its populations bounced off a cell in this step still owe their C
      // (the next sweep would have added it): C_r enters direction rbar,
      // momentum -C_r c_r, with the velocity of this step's half step at
      // the link's cell at its position of this step
      const float4 pu = lv.pu[idx];
      const uint32_t pm = __float_as_uint(pu.w);
      if (impulses) {
        float mf[3] = {0.f, 0.f, 0.f};
        for (int r = 0; r < Q; ++r) {
          const float v = Store<S>::ld(pop + slot[r]);
          mf[0] += v * D::cx(r);
          mf[1] += v * D::cy(r);
          mf[2] += v * D::cz(r);
        }
        // C_r owed to direction rbar: momentum -C_r c_r (the links to a second
        // or third cell got theirs in place)
        for (uint32_t m = pm; m; m &= m - 1u) {
          const int r = __ffs(m) - 1;
          const float cx = (float)rt_c<0>(r), cy = (float)rt_c<1>(r), cz = (float)rt_c<2>(r);
          const float C = -((float)rt_m(r) / 6.0f) * (cx * pu.x + cy * pu.y + cz * pu.z);
          mf[0] -= C * cx;
          mf[1] -= C * cy;
          mf[2] -= C * cz;
        }
        const double mom[3] = {mf[0], mf[1], mf[2]};
        const double tq[3] = {arm_n[1] * mom[2] - arm_n[2] * mom[1], arm_n[2] * mom[0] - arm_n[0] * mom[2],
                              arm_n[0] * mom[1] - arm_n[1] * mom[0]};
        atomic_add3(pv.PF + 3 * nw, mom);
        atomic_add3(pv.PT + 3 * nw, tq);
      }
      if (pm) reinterpret_cast<float *>(lv.pu + idx)[3] = 0.f;
    } else if (old >= 0) {
      const double mom[3] = {pv.rho0 * u_o[0], pv.rho0 * u_o[1], pv.rho0 * u_o[2]};
      const double tq[3] = {arm_o[1] * mom[2] - arm_o[2] * mom[1], arm_o[2] * mom[0] - arm_o[0] * mom[2],
                            arm_o[0] * mom[1] - arm_o[1] * mom[0]};
      const double mneg[3] = {-mom[0], -mom[1], -mom[2]}, tneg[3] = {-tq[0], -tq[1], -tq[2]};
      atomic_add3(pv.PF + 3 * old, mneg);
      atomic_add3(pv.PT + 3 * old, tneg);
      if (nw == FLUID) {
        // uncovered: new fluid at n^eq(rho_bar, u_rigid), stored shifted
        const float rho0 = (float)pv.rho0;
        const float uu = u_o[0] * u_o[0] + u_o[1] * u_o[1] + u_o[2] * u_o[2];
        for (int r = 0; r < Q; ++r) {
          const float cu = D::cx(r) * u_o[0] + D::cy(r) * u_o[1] + D::cz(r) * u_o[2];
          const float w = D::m(r) / 36.0f;
          Store<S>::st(pop + slot[r], rho0 * w * (cu * (3.0f + cu * (4.5f + 4.5f * cu)) - uu * (1.5f + 4.5f * cu)));
        }
      } else {
        // direct change of owner: uncover by the old, cover by the new (reading Q6)
        const double tq2[3] = {arm_n[1] * mom[2] - arm_n[2] * mom[1], arm_n[2] * mom[0] - arm_n[0] * mom[2],
                               arm_n[0] * mom[1] - arm_n[1] * mom[0]};
        atomic_add3(pv.PF + 3 * nw, mom);
        atomic_add3(pv.PT + 3 * nw, tq2);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// geometry of the step, incrementally.  After resolve, a node's neighbour
// word can differ from the last one only if its own owner or a neighbour's
// changed, and every change is in the change list.  The contact sums of a
// cell come from the nodes it owns, which lie inside its ellipsoid at its
// current position (a cell owns only nodes it covers); they are summed at
// the start of the next step, beside its sweep (the sweep needs only the
// neighbour words).

// neighbour word of node (x, y, z) from the owner map: for a fluid node bit 0,
// bit r neighbour x + c_r solid, NB_WALL / NB_CELL some solid neighbour is a
// wall / a cell; for a cell node its contact links (bit r: the neighbour is a
// wall node or another cell's); zero for wall nodes
__device__ __forceinline__ uint32_t node_word(const LatticeView &lv, int x, int y, int z, uint32_t &cellw) {
  using D = D3Q19;
  const unsigned nx = (unsigned)lv.nx, nxy = (unsigned)lv.nx * (unsigned)lv.ny;
  cellw = NBC_MIXED;
  const int xs[3] = {x == 0 ? lv.nx - 1 : x - 1, x, x == lv.nx - 1 ? 0 : x + 1};
  const int ys[3] = {y == 0 ? lv.ny - 1 : y - 1, y, y == lv.ny - 1 ? 0 : y + 1};
  const int zs[3] = {z == 0 ? lv.nz - 1 : z - 1, z, z == lv.nz - 1 ? 0 : z + 1};
  // the node's owner and its 18 neighbours' are requested together (one
  // memory round trip; a wall node's neighbour owners go unused)
  int on[Q];
  sfor<0, Q>([&](auto R) {
    constexpr int r = decltype(R)::value;
    on[r] = lv.owner[(unsigned)xs[1 + D::cx(r)] + nx * (unsigned)ys[1 + D::cy(r)] + nxy * (unsigned)zs[1 + D::cz(r)]];
  });
  const int own = on[0];
  if (own <= -2) return 0u;  // wall node
  if (own != FLUID) {
    // cell node: its contact links (neighbours owned by a wall or another cell)
    unsigned cmask = 0;
    sfor<1, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      cmask |= (on[r] != FLUID && on[r] != own ? 1u : 0u) << r;
    });
    return cmask;
  }
  unsigned solid = 0, wall = 0;
  int first = -1;
  bool mixed = false;
  sfor<1, Q>([&](auto R) {
    constexpr int r = decltype(R)::value;
    solid |= (on[r] != FLUID ? 1u : 0u) << r;
    wall |= (on[r] <= -2 ? 1u : 0u) << r;
    if (on[r] != FLUID) {
      if (first == -1) first = on[r];
      else if (on[r] != first) mixed = true;
    }
  });
  if (first >= 0 && !mixed) cellw = (uint32_t)first;
  return NB_FLUID | solid | (wall ? NB_WALL : 0u) | ((solid & ~wall) ? NB_CELL : 0u);
}

// neighbour words of every changed node x and of the nodes x - c_r that see
// it; the whole lattice if the change list overflowed (grid-stride)
__global__ void k_nbm_update(LatticeView lv, ChangeList chg) {
  using D = D3Q19;
  const int cnt = *chg.count;
  const bool all = cnt > chg.cap;
  const long long total = all ? (long long)lv.N : (long long)cnt * Q;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    int xyz[3];
    if (all) {
      node_xyz(lv, (unsigned)t, xyz);
    } else {
      const int c = (int)(t / Q), r = (int)(t - (long long)c * Q);
      node_xyz(lv, (unsigned)chg.items[3 * c], xyz);
      xyz[0] = wrapi(xyz[0] - D::cx(r), lv.nx);
      xyz[1] = wrapi(xyz[1] - D::cy(r), lv.ny);
      xyz[2] = wrapi(xyz[2] - D::cz(r), lv.nz);
    }
    uint32_t cw;
    const unsigned nn = node_of(lv, xyz[0], xyz[1], xyz[2]);
    lv.nbm[nn] = node_word(lv, xyz[0], xyz[1], xyz[2], cw);
    lv.nbc[nn] = cw;
  }
}

// contact sums of one cell (one block per cell, Eqs. deltapppp,
// deltapppm): the rows of the cell's box, each cut to the outer interval of
// its ellipsoid at its current position, flattened over the block; every
// node the cell owns adds its links into another cell or a wall to exact
// integer sums (the cell's bounce links come from the sweep's records)
constexpr int LB = 128;  // threads of a contact block (8 blocks fit an SM)

__global__ void __launch_bounds__(LB) k_contacts(LatticeView lv, PartView pv) {
  using D = D3Q19;
  __shared__ int sh_w[LB / 32 + 1];
  __shared__ int s_off[LB + 1], s_x0[LB], s_y[LB], s_z[LB];
  __shared__ int s_ci[LB / 32][6];
  const int p = blockIdx.x;
  const int lo1 = pv.box[6 * p + 1], lo2 = pv.box[6 * p + 2];
  const int by = pv.box[6 * p + 4] - lo1 + 1, bz = pv.box[6 * p + 5] - lo2 + 1;
  const int rows = (by > 0 && bz > 0) ? by * bz : 0;
  CellGeo g;
  cell_geo(pv, p, g);
  const float ip = (float)pv.inv_rperp2, kk = (float)(pv.inv_rpar2 - pv.inv_rperp2);
  const int imin = lv.per[0] ? -(lv.nx / 2) : -g.Xi[0];
  const int imax = lv.per[0] ? imin + lv.nx - 1 : lv.nx - 1 - g.Xi[0];
  const float4 k0 = pv.kin[3 * p], k1 = pv.kin[3 * p + 1], k2 = pv.kin[3 * p + 2];
  const int Xk[3] = {(int)k0.w, (int)k1.w, (int)k2.w};
  const unsigned nx = (unsigned)lv.nx, nxy = (unsigned)lv.nx * (unsigned)lv.ny;
  int ci[6] = {0, 0, 0, 0, 0, 0};
  for (int r0 = 0; r0 < rows; r0 += LB) {
    const int t = r0 + threadIdx.x;
    int len = 0, ao = 0, y = 0, z = 0;
    if (t < rows) {
      y = lo1 + t % by;
      z = lo2 + t / by;
      if (lv.per[1]) y = wrapi(y, lv.ny);
      if (lv.per[2]) z = wrapi(z, lv.nz);
      const RowQuad qn = row_quad((float)imin_image(y - g.Xi[1], lv.ny, lv.per[1]) - g.Xf[1],
                                  (float)imin_image(z - g.Xi[2], lv.nz, lv.per[2]) - g.Xf[2], g.of, ip, kk);
      int bo;
      row_range(qn, 1.0f + ROW_EPS, g.Xf[0], ao, bo);
      ao = max(ao, imin);
      bo = min(bo, imax);
      len = bo >= ao ? bo - ao + 1 : 0;
    }
    int tot;
    const int off = block_scan<LB>(len, sh_w, &tot);
    s_off[threadIdx.x] = off;
    s_x0[threadIdx.x] = ao;
    s_y[threadIdx.x] = y;
    s_z[threadIdx.x] = z;
    __syncthreads();
    for (int k = threadIdx.x; k < tot; k += LB) {
      // the row holding flattened node k: the last row starting at or before k
      int lo = 0, hi = LB - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_off[mid] <= k) lo = mid;
        else hi = mid - 1;
      }
      int x = g.Xi[0] + s_x0[lo] + (k - s_off[lo]);
      if (lv.per[0]) x = wrapi(x, lv.nx);
      const int yy = s_y[lo], zz = s_z[lo];
      const unsigned nn = (unsigned)x + nx * (unsigned)yy + nxy * (unsigned)zz;
      if (lv.owner[nn] != p) continue;
      // the node's contact links, kept in its neighbour word by the geometry passes
      const unsigned cmask = lv.nbm[nn] & NB_SOLID;
      if (cmask) {
        const int di[3] = {imin_image(x - Xk[0], lv.nx, lv.per[0]), imin_image(yy - Xk[1], lv.ny, lv.per[1]),
                           imin_image(zz - Xk[2], lv.nz, lv.per[2])};
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
    }
    __syncthreads();  // the row tables are rewritten by the next chunk
  }
  block_sum_i<6, LB>(ci, s_ci);
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) {
      pv.cK[3 * p + k] = ci[k];
      pv.cIT[3 * p + k] = ci[3 + k];
    }
}

// owners >= 0 become resting fluid (first particles_set), layout of parity par
template <class S>
__global__ void k_clear_cells(LatticeView lv, int par) {
  using D = D3Q19;
  const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= lv.N) return;
  if (lv.owner[n] < 0) return;
  lv.owner[n] = FLUID;
  int xyz[3];
  node_xyz(lv, n, xyz);
  S *pop = reinterpret_cast<S *>(lv.pop);
  for (int r = 0; r < Q; ++r) {
    unsigned slot;
    if (par == 0 || r == 0) slot = (unsigned)r * lv.N + n;
    else
      slot = (unsigned)D::opp(r) * lv.N +
             node_of(lv, wrapi(xyz[0] - D::cx(r), lv.nx), wrapi(xyz[1] - D::cy(r), lv.ny), wrapi(xyz[2] - D::cz(r), lv.nz));
    Store<S>::st(pop + slot, 0.0f);
  }
}

// ---------------------------------------------------------------------------
// learned near-contact correction: pair features, close pairs, application

// features of the ordered pair (i, j) in the body frame of i (R the rotation
// of i): R^T r, q_i^* q_j with w >= 0, the gap |r| - sigma_R (Eq. sigma with
// the fluid-coupling half-axes), R^T (V_j - V_i), R^T (W_j - W_i); velocities
// of the current kinematics
__device__ void pair_features(const LatticeView &lv, const PartView &pv, int i, int j, float f[14], float R[3][3]) {
  const float4 a0 = pv.kin[3 * i], a1 = pv.kin[3 * i + 1], a2 = pv.kin[3 * i + 2];
  const float4 b0 = pv.kin[3 * j], b1 = pv.kin[3 * j + 1], b2 = pv.kin[3 * j + 2];
  const int dims[3] = {lv.nx, lv.ny, lv.nz};
  const int ai[3] = {(int)a0.w, (int)a1.w, (int)a2.w}, bi[3] = {(int)b0.w, (int)b1.w, (int)b2.w};
  const float af[3] = {a0.x, a0.y, a0.z}, bf[3] = {b0.x, b0.y, b0.z};
  float r[3];
  for (int k = 0; k < 3; ++k) r[k] = (float)imin_image(bi[k] - ai[k], dims[k], lv.per[k]) + (bf[k] - af[k]);
  const double *qi = pv.q + 4 * i, *qj = pv.q + 4 * j;
  rotmat_f(qi, R);
  float Rj[3][3];
  rotmat_f(qj, Rj);
  const float oi[3] = {R[0][2], R[1][2], R[2][2]}, oj[3] = {Rj[0][2], Rj[1][2], Rj[2][2]};
  const float rl = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]), ir = 1.0f / rl;
  const float a = (r[0] * oi[0] + r[1] * oi[1] + r[2] * oi[2]) * ir, b = (r[0] * oj[0] + r[1] * oj[1] + r[2] * oj[2]) * ir;
  const float c = oi[0] * oj[0] + oi[1] * oj[1] + oi[2] * oj[2];
  const float Rp2 = (float)(pv.R_par * pv.R_par), Rq2 = (float)(pv.R_perp * pv.R_perp);
  const float chi = (Rp2 - Rq2) / (Rp2 + Rq2);
  const float S = 1.0f - 0.5f * chi * ((a + b) * (a + b) / (1.0f + chi * c) + (a - b) * (a - b) / (1.0f - chi * c));
  const float gap = rl - 2.0f * (float)pv.R_perp * rsqrtf(S);
  const float dv[3] = {b1.x - a1.x, b1.y - a1.y, b1.z - a1.z}, dw[3] = {b2.x - a2.x, b2.y - a2.y, b2.z - a2.z};
  for (int k = 0; k < 3; ++k) {
    f[k] = R[0][k] * r[0] + R[1][k] * r[1] + R[2][k] * r[2];
    f[8 + k] = R[0][k] * dv[0] + R[1][k] * dv[1] + R[2][k] * dv[2];
    f[11 + k] = R[0][k] * dw[0] + R[1][k] * dw[1] + R[2][k] * dw[2];
  }
  const float w1 = (float)qi[0], x1 = -(float)qi[1], y1 = -(float)qi[2], z1 = -(float)qi[3];
  const float w2 = (float)qj[0], x2 = (float)qj[1], y2 = (float)qj[2], z2 = (float)qj[3];
  float qr[4] = {w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                 w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2};
  const float sgn = qr[0] < 0.f ? -1.f : 1.f;
  for (int k = 0; k < 4; ++k) f[3 + k] = sgn * qr[k];
  f[7] = gap;
}

__global__ void k_pair_features(LatticeView lv, PartView pv, const int2 *pairs, int n, float *out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int2 pr = pairs[t];
  if (pr.x < 0 || pr.x >= pv.n || pr.y < 0 || pr.y >= pv.n || pr.x == pr.y) {
    for (int k = 0; k < 14; ++k) out[14 * t + k] = 0.f;
    return;
  }
  float f[14], R[3][3];
  pair_features(lv, pv, pr.x, pr.y, f, R);
  for (int k = 0; k < 14; ++k) out[14 * t + k] = f[k];
}

// close pairs (gap_lo <= gap < gap_cut, relative speed |V_j - V_i| in
// [speed_lo, speed_hi]) from the cell list, one block per cell
// (lane b < 27 scans bin b), with their features
__global__ void k_mlp_pairs(LatticeView lv, PartView pv, CellListView cl, PairBuf pb, float gap_lo, float gap_cut,
                            float speed_lo, float speed_hi) {
  const int i = blockIdx.x;
  if (threadIdx.x >= 27) return;
  const int bin = cl.bin_of[i];
  const int bc[3] = {bin % cl.nb[0], (bin / cl.nb[0]) % cl.nb[1], bin / (cl.nb[0] * cl.nb[1])};
  int off[3][3], noff[3];
  for (int k = 0; k < 3; ++k) noff[k] = bin_offsets(cl.nb[k], lv.per[k], bc[k], off[k]);
  const int ix = threadIdx.x % 3, iy = (threadIdx.x / 3) % 3, iz = threadIdx.x / 9;
  if (ix >= noff[0] || iy >= noff[1] || iz >= noff[2]) return;
  const int b = wrapi(bc[0] + off[0][ix], cl.nb[0]) +
                cl.nb[0] * (wrapi(bc[1] + off[1][iy], cl.nb[1]) + cl.nb[1] * wrapi(bc[2] + off[2][iz], cl.nb[2]));
  const int e = cl.start[b + 1];
  for (int k = cl.start[b]; k < e; ++k) {
    const int j = cl.ids[k];
    if (j == i) continue;
    float f[14], R[3][3];
    pair_features(lv, pv, i, j, f, R);
    if (!(f[7] >= gap_lo && f[7] < gap_cut)) continue;  // outside the range: the plain method
    const float sp = sqrtf(f[8] * f[8] + f[9] * f[9] + f[10] * f[10]);
    if (!(sp >= speed_lo && sp <= speed_hi)) continue;
    const int s = atomicAdd(pb.count, 1);
    if (s >= pb.cap) {
      atomicOr(pv.status, ST_OVERFLOW);
      continue;
    }
    pb.pairs[s] = make_int2(i, j);
    for (int q = 0; q < 14; ++q) pb.feat[14 * s + q] = f[q];
  }
}

// the network's force and torque on i, back from its body frame to the lab
// frame, added to the potentials of the step
__global__ void k_mlp_apply(PartView pv, PairBuf pb) {
  const int n = min(*pb.count, pb.cap);
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const int i = pb.pairs[s].x;
    float R[3][3];
    rotmat_f(pv.q + 4 * i, R);
    const float *y = pb.out + 6 * s;
    for (int k = 0; k < 3; ++k) {
      atomicAdd(&pv.Fpot[3 * i + k], (double)(R[k][0] * y[0] + R[k][1] * y[1] + R[k][2] * y[2]));
      atomicAdd(&pv.Tpot[3 * i + k], (double)(R[k][0] * y[3] + R[k][1] * y[4] + R[k][2] * y[5]));
    }
  }
}

// ---------------------------------------------------------------------------
// host-side launchers

static inline unsigned nblk(unsigned n, unsigned b) { return (n + b - 1) / b; }

void launch_cell_list(const LatticeView &lv, const PartView &pv, const CellListView &cl, cudaStream_t st, int64_t *nl) {
  if (pv.n == 0) return;
  k_cl_bin<<<nblk(pv.n, 128), 128, 0, st>>>(lv, pv, cl);
  k_cl_scan<<<1, 1024, 0, st>>>(cl);
  k_cl_scatter<<<nblk(pv.n, 128), 128, 0, st>>>(pv, cl);
  k_cl_sort<<<nblk(cl.nbins, 128), 128, 0, st>>>(cl);
  *nl += 4;
}

void launch_forces(const LatticeView &lv, const PartView &pv, const CellListView &cl, const SurfBits &sb,
                   cudaStream_t st, int64_t *nl) {
  if (pv.n == 0) return;
  k_forces<<<pv.n, FB, 0, st>>>(lv, pv, cl, sb);
  *nl += 1;
}

void launch_sums_solve(int dtype, const LatticeView &lv, const PartView &pv, int par, cudaStream_t st, int64_t *nl) {
  (void)dtype;
  (void)par;
  if (pv.n == 0) return;
  k_link_reduce<<<pv.n, LT, 0, st>>>(lv, pv);
  k_solve<<<nblk(pv.n, BL_SOLVE_TB), BL_SOLVE_TB, 0, st>>>(lv, pv);
  *nl += 2;
}

void launch_link_pending(int dtype, const LatticeView &lv, const PartView &pv, int par, cudaStream_t st,
                         int64_t *nl) {
  if (pv.n == 0) return;
  if (dtype == 0) k_link_pending<float><<<pv.n, LT, 0, st>>>(lv, pv, par);
  else if (dtype == 1) k_link_pending<__nv_bfloat16><<<pv.n, LT, 0, st>>>(lv, pv, par);
  else k_link_pending<__half><<<pv.n, LT, 0, st>>>(lv, pv, par);
  *nl += 1;
}

void launch_flush_pending(int dtype, const LatticeView &lv, int par, cudaStream_t st, int64_t *nl) {
  const unsigned b = 256, g = nblk(lv.N, b) < 4u * 152u ? nblk(lv.N, b) : 4u * 152u;
  if (dtype == 0) k_flush_pending<float><<<g, b, 0, st>>>(lv, par);
  else if (dtype == 1) k_flush_pending<__nv_bfloat16><<<g, b, 0, st>>>(lv, par);
  else k_flush_pending<__half><<<g, b, 0, st>>>(lv, par);
  *nl += 1;
}

void launch_pair_features(const LatticeView &lv, const PartView &pv, const int2 *pairs, int n, float *out,
                          cudaStream_t st) {
  if (n > 0) k_pair_features<<<nblk(n, 128), 128, 0, st>>>(lv, pv, pairs, n, out);
}

void launch_mlp_correction(const LatticeView &lv, const PartView &pv, const CellListView &cl, const PairBuf &pb,
                           float gap_lo, float gap_cut, float speed_lo, float speed_hi, const void *mlp,
                           cudaStream_t st, int64_t *nl) {
  if (pv.n == 0) return;
  cudaMemsetAsync(pb.count, 0, sizeof(int), st);
  k_mlp_pairs<<<pv.n, 32, 0, st>>>(lv, pv, cl, pb, gap_lo, gap_cut, speed_lo, speed_hi);
  launch_mlp_forward_dev(mlp, pb.feat, pb.count, pb.cap, pb.out, st);
  k_mlp_apply<<<nblk((unsigned)pb.cap, 128) < 152u ? nblk((unsigned)pb.cap, 128) : 152u, 128, 0, st>>>(pv, pb);
  *nl += 3;
}

void launch_set_state(const LatticeView &lv, const PartView &pv, int mode, cudaStream_t st, int64_t *nl) {
  if (pv.n == 0) return;
  k_set_state<<<nblk(pv.n, 64), 64, 0, st>>>(lv, pv, mode);
  *nl += 1;
}

void launch_claims(const LatticeView &lv, const PartView &pv, int *claim, const ChangeList &chg, int mode,
                   cudaStream_t st, int64_t *nl) {
  if (pv.n == 0) return;
  k_claims<<<pv.n, PB, 0, st>>>(lv, pv, claim, chg, mode);
  *nl += 1;
}

void launch_nbm_update(const LatticeView &lv, const PartView &pv, const ChangeList &chg, cudaStream_t st,
                       int64_t *nl) {
  if (pv.n == 0) return;
  k_nbm_update<<<4 * 152, 256, 0, st>>>(lv, chg);
  *nl += 1;
}

void launch_contacts(const LatticeView &lv, const PartView &pv, cudaStream_t st, int64_t *nl) {
  if (pv.n == 0) return;
  k_contacts<<<pv.n, LB, 0, st>>>(lv, pv);
  *nl += 1;
}

void launch_resolve_fill(int dtype, const LatticeView &lv, const PartView &pv, const CellListView &cl, int *claim,
                         const ChangeList &chg, int par_next, int impulses, cudaStream_t st, int64_t *nl) {
  if (pv.n == 0) return;
  if (dtype == 0) k_resolve_fill<float><<<pv.n, PB, 0, st>>>(lv, pv, cl, claim, chg, par_next, impulses);
  else if (dtype == 1) k_resolve_fill<__nv_bfloat16><<<pv.n, PB, 0, st>>>(lv, pv, cl, claim, chg, par_next, impulses);
  else k_resolve_fill<__half><<<pv.n, PB, 0, st>>>(lv, pv, cl, claim, chg, par_next, impulses);
  *nl += 1;
}


void launch_clear_cells(int dtype, const LatticeView &lv, int par, cudaStream_t st, int64_t *nl) {
  const unsigned b = 256, g = nblk(lv.N, b);
  if (dtype == 0) k_clear_cells<float><<<g, b, 0, st>>>(lv, par);
  else if (dtype == 1) k_clear_cells<__nv_bfloat16><<<g, b, 0, st>>>(lv, par);
  else k_clear_cells<__half><<<g, b, 0, st>>>(lv, par);
  *nl += 1;
}

}  // namespace bl
