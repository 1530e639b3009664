// particle_kernels.cu -- the cell side of the coupled step (arXiv:1005.2594):
//
//   cell list      count -> scan -> scatter -> per-bin sort, canonical (bin, id)
//   potentials     Berne-Pechukas-scaled Hookean cell-cell pairs (Sec. III,
//                  Eqs. phi, epsilon, sigma) and cell-wall spheres (Eq. sigmaw),
//                  one warp per cell, FP32 arithmetic, FP64 result
//   leap-frog      V, X and the lab-frame angular momentum L, exact quaternion
//                  exponential (Sec. II; reading Q4), FP64, one block per cell;
//                  the same block then claims the nodes its new ellipsoid covers
//   resolve        first-arrival owner rule (Sec. II single occupancy), then
//                  fill/drain of every changed node with the momentum balance
//                  given to the cells (Sec. II)
//
// Ownership claims.  claim[] holds INT_MAX ("untouched") on every node
// between steps.  In the claim pass each cell visits the nodes of the box
// that holds both its old and its new ellipsoid: the current owner marks a
// node it still covers with KEEP (INT_MIN) and one it leaves with TOUCHED
// (INT_MAX - 1); any other cell covering the node writes its index; all
// with atomicMin.  In the resolve pass the first visitor of a node takes the
// claim with atomicExch(INT_MAX) and decodes: KEEP -> old owner, TOUCHED ->
// fluid, a cell index -> the lowest index that newly covers the node.
#include <climits>

#include "bl_internal.cuh"

namespace bl {

constexpr int CLAIM_FREE = INT_MAX;
constexpr int CLAIM_TOUCHED = INT_MAX - 1;
constexpr int CLAIM_KEEP = INT_MIN;

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

// cell-cell pair, force and torque on i; r = X_j - X_i
__device__ __forceinline__ void bp_pair(const float r[3], const float oi[3], const float oj[3], const PartView &pv,
                                        float F[3], float T[3]) {
  const float r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  if (!(r2 > 0.f)) return;
  const float rl = sqrtf(r2), ir = 1.0f / rl;
  const float rh[3] = {r[0] * ir, r[1] * ir, r[2] * ir};
  const float a = rh[0] * oi[0] + rh[1] * oi[1] + rh[2] * oi[2];
  const float b = rh[0] * oj[0] + rh[1] * oj[1] + rh[2] * oj[2];
  const float c = oi[0] * oj[0] + oi[1] * oj[1] + oi[2] * oj[2];
  const float chi = pv.chi;
  const float ap = a + b, am = a - b;
  const float dp = 1.0f + chi * c, dm = 1.0f - chi * c;
  const float S = 1.0f - 0.5f * chi * (ap * ap / dp + am * am / dm);
  const float sigma = pv.sigbar * rsqrtf(S);
  if (rl >= sigma) return;
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
  const float h = 1.0f - rl / sigma;
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

// cell-wall sphere, force and torque on the cell; r = x_wall - X
__device__ __forceinline__ void bp_wall(const float r[3], const float oi[3], const PartView &pv, float F[3], float T[3]) {
  const float r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  if (!(r2 > 0.f) || r2 >= pv.sigw_max * pv.sigw_max) return;
  const float rl = sqrtf(r2), ir = 1.0f / rl;
  const float rh[3] = {r[0] * ir, r[1] * ir, r[2] * ir};
  const float a = rh[0] * oi[0] + rh[1] * oi[1] + rh[2] * oi[2];
  const float D = 1.0f - pv.chi_w * a * a;
  const float sigma = pv.sigbar_w * rsqrtf(D);
  if (rl >= sigma) return;
  const float eps = pv.eps_w;
  const float h = 1.0f - rl / sigma;
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

__global__ void __launch_bounds__(128) k_forces(LatticeView lv, PartView pv, CellListView cl, WallRows wr) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= pv.n) return;
  const float4 a0 = pv.kin[3 * i], a1 = pv.kin[3 * i + 1], a2 = pv.kin[3 * i + 2];
  const int Xi[3] = {(int)a0.w, (int)a1.w, (int)a2.w};
  const float fi[3] = {a0.x, a0.y, a0.z};
  const float oi[3] = {(float)pv.o[3 * i], (float)pv.o[3 * i + 1], (float)pv.o[3 * i + 2]};
  const int dims[3] = {lv.nx, lv.ny, lv.nz};
  float F[3] = {0.f, 0.f, 0.f}, T[3] = {0.f, 0.f, 0.f};
  // pairs over the neighbouring bins
  const int bin = cl.bin_of[i];
  const int bc[3] = {bin % cl.nb[0], (bin / cl.nb[0]) % cl.nb[1], bin / (cl.nb[0] * cl.nb[1])};
  int off[3][3], noff[3];
  for (int k = 0; k < 3; ++k) noff[k] = bin_offsets(cl.nb[k], lv.per[k], bc[k], off[k]);
  const float rc2 = pv.r_cut * pv.r_cut;
  for (int iz = 0; iz < noff[2]; ++iz)
    for (int iy = 0; iy < noff[1]; ++iy)
      for (int ix = 0; ix < noff[0]; ++ix) {
        const int bx = wrapi(bc[0] + off[0][ix], cl.nb[0]);
        const int by = wrapi(bc[1] + off[1][iy], cl.nb[1]);
        const int bz = wrapi(bc[2] + off[2][iz], cl.nb[2]);
        const int b = bx + cl.nb[0] * (by + cl.nb[1] * bz);
        const int e = cl.start[b + 1];
        for (int k = cl.start[b] + lane; k < e; k += 32) {
          const int j = cl.ids[k];
          if (j == i) continue;
          const float4 b0 = pv.kin[3 * j], b1 = pv.kin[3 * j + 1], b2 = pv.kin[3 * j + 2];
          const int Xj[3] = {(int)b0.w, (int)b1.w, (int)b2.w};
          const float fj[3] = {b0.x, b0.y, b0.z};
          float r[3];
          for (int m = 0; m < 3; ++m) r[m] = (float)imin_image(Xj[m] - Xi[m], dims[m], lv.per[m]) + (fj[m] - fi[m]);
          if (r[0] * r[0] + r[1] * r[1] + r[2] * r[2] >= rc2) continue;
          const float oj[3] = {(float)pv.o[3 * j], (float)pv.o[3 * j + 1], (float)pv.o[3 * j + 2]};
          bp_pair(r, oi, oj, pv, F, T);
        }
      }
  // surface wall nodes in the rows of the box around the cell
  if (wr.row_start) {
    const int R = (int)ceilf(pv.sigw_max) + 1;
    const int side = 2 * R + 1;
    for (int t = lane; t < side * side; t += 32) {
      int y = Xi[1] - R + t % side, z = Xi[2] - R + t / side;
      if (lv.per[1]) y = wrapi(y, lv.ny);
      else if (y < 0 || y >= lv.ny) continue;
      if (lv.per[2]) z = wrapi(z, lv.nz);
      else if (z < 0 || z >= lv.nz) continue;
      const int row = y + lv.ny * z;
      const int s = wr.row_start[row], e = wr.row_start[row + 1];
      if (s == e) continue;
      const float ry = (float)imin_image(y - Xi[1], lv.ny, lv.per[1]) - fi[1];
      const float rz = (float)imin_image(z - Xi[2], lv.nz, lv.per[2]) - fi[2];
      if (ry * ry + rz * rz >= pv.sigw_max * pv.sigw_max) continue;
      // x range [Xi - R, Xi + R], split where it wraps
      int ra[3], rb[3], nr = 0;
      const int xlo = Xi[0] - R, xhi = Xi[0] + R;
      if (2 * R + 1 >= lv.nx) {
        ra[0] = 0; rb[0] = lv.nx - 1; nr = 1;
      } else if (!lv.per[0]) {
        ra[0] = max(xlo, 0); rb[0] = min(xhi, lv.nx - 1); nr = 1;
      } else {
        ra[nr] = max(xlo, 0); rb[nr] = min(xhi, lv.nx - 1); ++nr;
        if (xlo < 0) { ra[nr] = xlo + lv.nx; rb[nr] = lv.nx - 1; ++nr; }
        if (xhi >= lv.nx) { ra[nr] = 0; rb[nr] = xhi - lv.nx; ++nr; }
      }
      for (int q = 0; q < nr; ++q) {
        int lo = s, hi = e;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (wr.row_x[mid] < ra[q]) lo = mid + 1;
          else hi = mid;
        }
        for (int k = lo; k < e && wr.row_x[k] <= rb[q]; ++k) {
          const int xw = wr.row_x[k];
          const float rx = (float)imin_image(xw - Xi[0], lv.nx, lv.per[0]) - fi[0];
          const float r[3] = {rx, ry, rz};
          bp_wall(r, oi, pv, F, T);
        }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    F[m] = warp_sum(F[m]);
    T[m] = warp_sum(T[m]);
  }
  if (lane == 0)
    for (int m = 0; m < 3; ++m) {
      pv.Fpot[3 * i + m] = (double)F[m];
      pv.Tpot[3 * i + m] = (double)T[m];
    }
}

// ---------------------------------------------------------------------------
// leap-frog and claims

__device__ void omega_from_L(const PartView &pv, const double q[4], const double L[3], double Om[3]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  double R[3][3];
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
  double Lb[3];
  for (int i = 0; i < 3; ++i) Lb[i] = R[0][i] * L[0] + R[1][i] * L[1] + R[2][i] * L[2];
  const double wb[3] = {Lb[0] / pv.Iperp, Lb[1] / pv.Iperp, Lb[2] / pv.Ipar};
  for (int i = 0; i < 3; ++i) Om[i] = R[i][0] * wb[0] + R[i][1] * wb[1] + R[i][2] * wb[2];
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

__device__ void aabb(const PartView &pv, const double X[3], const double o[3], int lo[3], int hi[3]) {
  for (int k = 0; k < 3; ++k) {
    const double h = sqrt(pv.R_perp * pv.R_perp * (1.0 - o[k] * o[k]) + pv.R_par * pv.R_par * o[k] * o[k]) + 0.01;
    lo[k] = (int)floor(X[k] - h);
    hi[k] = (int)ceil(X[k] + h);
  }
}

__device__ void inertia_lab(const PartView &pv, const double q[4], double I[3][3]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  double R[3][3];
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
  const double d[3] = {pv.Iperp, pv.Iperp, pv.Ipar};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) I[i][j] = R[i][0] * d[0] * R[j][0] + R[i][1] * d[1] * R[j][1] + R[i][2] * d[2] * R[j][2];
}

// A x = b, A symmetric positive definite 6 x 6 (Cholesky)
__device__ void solve_spd6(double A[6][6], const double b[6], double x[6]) {
  for (int j = 0; j < 6; ++j) {
    double d = A[j][j];
    for (int k = 0; k < j; ++k) d -= A[j][k] * A[j][k];
    d = sqrt(d);
    A[j][j] = d;
    for (int i = j + 1; i < 6; ++i) {
      double v = A[i][j];
      for (int k = 0; k < j; ++k) v -= A[i][k] * A[j][k];
      A[i][j] = v / d;
    }
  }
  double y[6];
  for (int i = 0; i < 6; ++i) {
    double v = b[i];
    for (int k = 0; k < i; ++k) v -= A[i][k] * y[k];
    y[i] = v / A[i][i];
  }
  for (int i = 5; i >= 0; --i) {
    double v = y[i];
    for (int k = i + 1; k < 6; ++k) v -= A[k][i] * x[k];
    x[i] = v / A[i][i];
  }
}

// inside test: FP32 filter, exact FP64 re-evaluation within 1e-3 of the surface
__device__ __forceinline__ bool inside_cell(int x, int y, int z, const double *X, const double *o, const float *Xf,
                                            const int *Xi, const float *of, const PartView &pv, const LatticeView &lv) {
  const float d0 = (float)imin_image(x - Xi[0], lv.nx, lv.per[0]) - Xf[0];
  const float d1 = (float)imin_image(y - Xi[1], lv.ny, lv.per[1]) - Xf[1];
  const float d2 = (float)imin_image(z - Xi[2], lv.nz, lv.per[2]) - Xf[2];
  const float dpar = d0 * of[0] + d1 * of[1] + d2 * of[2];
  const float dd = d0 * d0 + d1 * d1 + d2 * d2;
  const float s = dpar * dpar * (float)pv.inv_rpar2 + (dd - dpar * dpar) * (float)pv.inv_rperp2;
  if (fabsf(s - 1.0f) >= 1e-3f) return s < 1.0f;
  return inside_exact(x, y, z, X, o, pv.inv_rpar2, pv.inv_rperp2, lv);
}

// mode 0: time step (integrate, then claim if cells move)
// mode 1: first particles_set (state from stage, every old owner is fluid)
// mode 2: later particles_set (state from stage, first-arrival claims)
__global__ void __launch_bounds__(256) k_integrate_claim(LatticeView lv, PartView pv, int *claim, ChangeList chg,
                                                         int mode) {
  const int p = blockIdx.x;
  __shared__ double sX[3], so[3];
  __shared__ int slo[3], shi[3];
  __shared__ int sactive;
  if (threadIdx.x == 0) {
    if (p == 0) *chg.count = 0;
    double X[3], q[4], V[3], L[3], Om[3], o_old[3];
    for (int k = 0; k < 3; ++k) {
      X[k] = pv.X[3 * p + k];
      V[k] = pv.V[3 * p + k];
      L[k] = pv.L[3 * p + k];
      Om[k] = pv.Om[3 * p + k];
    }
    for (int k = 0; k < 4; ++k) q[k] = pv.q[4 * p + k];
    const double Xold[3] = {X[0], X[1], X[2]};
    axis_exact(q, o_old);
    bool moved = true;
    if (mode == 0) {
      // link force: variable part (FP64 sums) + constant part from the exact
      // integer sums, with f = X - rint(X) the fractional part the sweep used
      const double c = pv.rho0 / 18.0;
      double f[3], K[3], IT[3], Fl[3], Tl[3];
      for (int k = 0; k < 3; ++k) {
        f[k] = X[k] - rint(X[k]);
        K[k] = (double)pv.acc.K[3 * p + k];
        IT[k] = (double)pv.acc.IT[3 * p + k];
      }
      const double fxK[3] = {f[1] * K[2] - f[2] * K[1], f[2] * K[0] - f[0] * K[2], f[0] * K[1] - f[1] * K[0]};
      double Ft[3], Tt[3];
      for (int k = 0; k < 3; ++k) {
        Fl[k] = pv.acc.F[3 * p + k] + c * K[k];
        Tl[k] = pv.acc.T[3 * p + k] + c * (IT[k] - fxK[k]);
        Ft[k] = Fl[k] + pv.Fpot[3 * p + k] + pv.PF[3 * p + k] + (pv.bfc ? pv.m * pv.g[k] : 0.0);
        Tt[k] = Tl[k] + pv.Tpot[3 * p + k] + pv.PT[3 * p + k];
        pv.Flink[3 * p + k] = Fl[k];
        pv.Tlink[3 * p + k] = Tl[k];
        pv.Ftot[3 * p + k] = Ft[k];
        pv.Ttot[3 * p + k] = Tt[k];
        pv.acc.F[3 * p + k] = 0.0;
        pv.acc.T[3 * p + k] = 0.0;
        pv.acc.K[3 * p + k] = 0;
        pv.acc.IT[3 * p + k] = 0;
        pv.PF[3 * p + k] = 0.0;
        pv.PT[3 * p + k] = 0.0;
      }
      moved = pv.move != 0;
      if (moved) {
        // half-step velocities (reading Q3): the sweep bounced with the
        // predictor (Vp, Wp) of the kinematics; the link force at (V, W) is
        // F_link - Zff dV - Zft dW, dV = V - Vp, dW = W - Wp, and
        //   (m + Zff) dV + Zft dW = F_tot - m (Vp - V(t-1/2))
        //   Ztf dV + (I + Ztt) dW = T_tot + L(t-1/2) - I Wp
        const float4 k1 = pv.kin[3 * p + 1], k2 = pv.kin[3 * p + 2];
        const double Vp[3] = {k1.x, k1.y, k1.z}, Wp[3] = {k2.x, k2.y, k2.z};
        double I[3][3], Z[6][6], A[6][6], rhs[6], d[6];
        inertia_lab(pv, q, I);
        const double *z = pv.zeta + 21 * p;
        int k = 0;
        for (int a = 0; a < 3; ++a)
          for (int b = a; b < 3; ++b, ++k) Z[a][b] = Z[b][a] = z[k];
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b, ++k) Z[a][3 + b] = Z[3 + b][a] = z[k];
        for (int a = 0; a < 3; ++a)
          for (int b = a; b < 3; ++b, ++k) Z[3 + a][3 + b] = Z[3 + b][3 + a] = z[k];
        for (int a = 0; a < 6; ++a)
          for (int b = 0; b < 6; ++b) A[a][b] = Z[a][b];
        for (int a = 0; a < 3; ++a) {
          A[a][a] += pv.m;
          for (int b = 0; b < 3; ++b) A[3 + a][3 + b] += I[a][b];
          rhs[a] = Ft[a] - pv.m * (Vp[a] - V[a]);
          rhs[3 + a] = Tt[a] + L[a] - (I[a][0] * Wp[0] + I[a][1] * Wp[1] + I[a][2] * Wp[2]);
        }
        solve_spd6(A, rhs, d);
        for (int a = 0; a < 21; ++a) pv.zeta[21 * p + a] = 0.0;
        for (int a = 0; a < 6; ++a) pv.dvel[6 * p + a] = (float)d[a];
        // the link force at the solved velocities, and the totals of the step
        for (int a = 0; a < 3; ++a) {
          double dF = 0.0, dT = 0.0;
          for (int b = 0; b < 6; ++b) {
            dF += Z[a][b] * d[b];
            dT += Z[3 + a][b] * d[b];
          }
          Fl[a] -= dF;
          Tl[a] -= dT;
          Ft[a] -= dF;
          Tt[a] -= dT;
          pv.Flink[3 * p + a] = Fl[a];
          pv.Tlink[3 * p + a] = Tl[a];
          pv.Ftot[3 * p + a] = Ft[a];
          pv.Ttot[3 * p + a] = Tt[a];
          V[a] = Vp[a] + d[a];
          Om[a] = Wp[a] + d[3 + a];
        }
        for (int a = 0; a < 3; ++a) L[a] = I[a][0] * Om[0] + I[a][1] * Om[1] + I[a][2] * Om[2];
        const int dims[3] = {lv.nx, lv.ny, lv.nz};
        for (int a = 0; a < 3; ++a) {
          X[a] += V[a];
          if (lv.per[a]) {
            if (X[a] < 0.0) X[a] += (double)dims[a];
            else if (X[a] >= (double)dims[a]) X[a] -= (double)dims[a];
          }
        }
        const double th = sqrt(Om[0] * Om[0] + Om[1] * Om[1] + Om[2] * Om[2]);
        double dq[4] = {1.0, 0.0, 0.0, 0.0};
        if (th > 0.0) {
          double sn, cs;
          sincos(0.5 * th, &sn, &cs);
          const double sh = sn / th;
          dq[0] = cs;
          dq[1] = Om[0] * sh;
          dq[2] = Om[1] * sh;
          dq[3] = Om[2] * sh;
        }
        double nq[4];
        nq[0] = dq[0] * q[0] - dq[1] * q[1] - dq[2] * q[2] - dq[3] * q[3];
        nq[1] = dq[0] * q[1] + dq[1] * q[0] + dq[2] * q[3] - dq[3] * q[2];
        nq[2] = dq[0] * q[2] - dq[1] * q[3] + dq[2] * q[0] + dq[3] * q[1];
        nq[3] = dq[0] * q[3] + dq[1] * q[2] - dq[2] * q[1] + dq[3] * q[0];
        const double nn = sqrt(nq[0] * nq[0] + nq[1] * nq[1] + nq[2] * nq[2] + nq[3] * nq[3]);
        for (int k = 0; k < 4; ++k) q[k] = nq[k] / nn;
      }
    } else {
      const double *st = pv.stage + 13 * p;
      for (int k = 0; k < 3; ++k) {
        X[k] = st[k];
        V[k] = st[7 + k];
        L[k] = st[10 + k];
      }
      for (int k = 0; k < 4; ++k) q[k] = st[3 + k];
      omega_from_L(pv, q, L, Om);
    }
    for (int k = 0; k < 3; ++k) {
      pv.X[3 * p + k] = X[k];
      pv.V[3 * p + k] = V[k];
      pv.L[3 * p + k] = L[k];
      pv.Om[3 * p + k] = Om[k];
    }
    for (int k = 0; k < 4; ++k) pv.q[4 * p + k] = q[k];
    double o_new[3];
    axis_exact(q, o_new);
    for (int k = 0; k < 3; ++k) pv.o[3 * p + k] = o_new[k];
    write_kin(pv, p, X, V, Om);
    bool finite = true;
    for (int k = 0; k < 3; ++k)
      finite = finite && isfinite(X[k]) && isfinite(o_new[k]) && (mode == 1 || (isfinite(Xold[k]) && isfinite(o_old[k])));
    if (!finite) {
      // a non-finite state is reported and its box left empty
      atomicOr(pv.status, ST_UNSTABLE);
      for (int k = 0; k < 3; ++k) {
        pv.box[6 * p + k] = 0;
        pv.box[6 * p + 3 + k] = -1;
        slo[k] = 0;
        shi[k] = -1;
      }
      sactive = 0;
    } else {
      int lo[3], hi[3], lo2[3], hi2[3];
      aabb(pv, X, o_new, lo, hi);
      if (mode != 1) {
        aabb(pv, Xold, o_old, lo2, hi2);
        for (int k = 0; k < 3; ++k) {
          lo[k] = min(lo[k], lo2[k]);
          hi[k] = max(hi[k], hi2[k]);
        }
      }
      const int dims[3] = {lv.nx, lv.ny, lv.nz};
      for (int k = 0; k < 3; ++k) {
        if (!lv.per[k]) {
          lo[k] = max(lo[k], 0);
          hi[k] = min(hi[k], dims[k] - 1);
        } else if (hi[k] - lo[k] + 1 > dims[k]) {
          lo[k] = 0;
          hi[k] = dims[k] - 1;
        }
        pv.box[6 * p + k] = lo[k];
        pv.box[6 * p + 3 + k] = hi[k];
        slo[k] = lo[k];
        shi[k] = hi[k];
        sX[k] = X[k];
        so[k] = o_new[k];
      }
      sactive = moved ? 1 : 0;
      if (!moved) pv.box[6 * p + 3] = pv.box[6 * p] - 1;  // empty box: nothing to resolve
    }
  }
  __syncthreads();
  if (!sactive) return;
  double X[3] = {sX[0], sX[1], sX[2]}, o[3] = {so[0], so[1], so[2]};
  int Xi[3];
  float Xf[3], of[3];
  for (int k = 0; k < 3; ++k) {
    Xi[k] = (int)rint(X[k]);
    Xf[k] = (float)(X[k] - (double)Xi[k]);
    of[k] = (float)o[k];
  }
  const int bx = shi[0] - slo[0] + 1, by = shi[1] - slo[1] + 1, bz = shi[2] - slo[2] + 1;
  const int total = (bx > 0 && by > 0 && bz > 0) ? bx * by * bz : 0;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int x = slo[0] + t % bx, y = slo[1] + (t / bx) % by, z = slo[2] + t / (bx * by);
    if (lv.per[0]) x = wrapi(x, lv.nx);
    if (lv.per[1]) y = wrapi(y, lv.ny);
    if (lv.per[2]) z = wrapi(z, lv.nz);
    const unsigned idx = (unsigned)x + (unsigned)lv.nx * ((unsigned)y + (unsigned)lv.ny * z);
    const int ow = lv.owner[idx];
    if (ow <= -2) continue;
    const bool ins = inside_cell(x, y, z, X, o, Xf, Xi, of, pv, lv);
    if (mode == 1) {
      if (ins) atomicMin(&claim[idx], p);
    } else if (ow == p) {
      atomicMin(&claim[idx], ins ? CLAIM_KEEP : CLAIM_TOUCHED);
    } else if (ins) {
      atomicMin(&claim[idx], p);
    }
  }
}

// ---------------------------------------------------------------------------
// resolve + fill/drain

template <class S>
__device__ void node_slots(const LatticeView &lv, int par, int x, int y, int z, unsigned slot[Q]) {
  using D = D3Q19;
  const unsigned n = (unsigned)x + (unsigned)lv.nx * ((unsigned)y + (unsigned)lv.ny * z);
  for (int r = 0; r < Q; ++r) {
    if (par == 0 || r == 0) {
      slot[r] = (unsigned)r * lv.N + n;
    } else {
      const int xs = wrapi(x - D::cx(r), lv.nx), ys = wrapi(y - D::cy(r), lv.ny), zs = wrapi(z - D::cz(r), lv.nz);
      slot[r] = (unsigned)D::opp(r) * lv.N + (unsigned)xs + (unsigned)lv.nx * ((unsigned)ys + (unsigned)lv.ny * zs);
    }
  }
}

__device__ __forceinline__ void atomic_add3(double *a, const double v[3]) {
  atomicAdd(a, v[0]);
  atomicAdd(a + 1, v[1]);
  atomicAdd(a + 2, v[2]);
}

template <class S>
__global__ void __launch_bounds__(256) k_resolve_fill(LatticeView lv, PartView pv, int *claim, ChangeList chg,
                                                       LinkList ll, int par_next, int impulses) {
  using D = D3Q19;
  const int p = blockIdx.x;
  if (p == 0 && threadIdx.x == 0) *ll.count = 0;  // the step's link list has been used
  const int lo[3] = {pv.box[6 * p], pv.box[6 * p + 1], pv.box[6 * p + 2]};
  const int hi[3] = {pv.box[6 * p + 3], pv.box[6 * p + 4], pv.box[6 * p + 5]};
  const int bx = hi[0] - lo[0] + 1, by = hi[1] - lo[1] + 1, bz = hi[2] - lo[2] + 1;
  if (bx <= 0 || by <= 0 || bz <= 0) return;
  const int total = bx * by * bz;
  const int lane = threadIdx.x & 31;
  S *pop = reinterpret_cast<S *>(lv.pop);
  const int dims[3] = {lv.nx, lv.ny, lv.nz};
  for (int base = 0; base < total; base += blockDim.x) {
    const int t = base + threadIdx.x;
    int x = 0, y = 0, z = 0, old = 0, nw = 0;
    bool changed = false;
    unsigned idx = 0;
    if (t < total) {
      x = lo[0] + t % bx;
      y = lo[1] + (t / bx) % by;
      z = lo[2] + t / (bx * by);
      if (lv.per[0]) x = wrapi(x, lv.nx);
      if (lv.per[1]) y = wrapi(y, lv.ny);
      if (lv.per[2]) z = wrapi(z, lv.nz);
      idx = (unsigned)x + (unsigned)lv.nx * ((unsigned)y + (unsigned)lv.ny * z);
      const int c = atomicExch(&claim[idx], CLAIM_FREE);
      if (c != CLAIM_FREE) {
        old = lv.owner[idx];
        nw = c == CLAIM_KEEP ? old : (c == CLAIM_TOUCHED ? FLUID : c);
        changed = nw != old;
        if (changed) lv.owner[idx] = nw;
      }
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
    const double xyz[3] = {(double)x, (double)y, (double)z};
    unsigned slot[Q];
    node_slots<S>(lv, par_next, x, y, z, slot);
    double arm_o[3] = {0, 0, 0}, u_o[3] = {0, 0, 0}, arm_n[3] = {0, 0, 0};
    if (old >= 0) {
      for (int k = 0; k < 3; ++k) arm_o[k] = min_image_exact(xyz[k] - pv.X[3 * old + k], dims[k], lv.per[k]);
      const double *W = pv.Om + 3 * old;
      u_o[0] = pv.V[3 * old + 0] + (W[1] * arm_o[2] - W[2] * arm_o[1]);
      u_o[1] = pv.V[3 * old + 1] + (W[2] * arm_o[0] - W[0] * arm_o[2]);
      u_o[2] = pv.V[3 * old + 2] + (W[0] * arm_o[1] - W[1] * arm_o[0]);
    }
    if (nw >= 0)
      for (int k = 0; k < 3; ++k) arm_n[k] = min_image_exact(xyz[k] - pv.X[3 * nw + k], dims[k], lv.per[k]);
    if (old == FLUID && nw >= 0) {
      // covered: the fluid is deleted, its momentum goes to the new owner
      if (impulses) {
        double mom[3] = {0, 0, 0};
        for (int r = 0; r < Q; ++r) {
          const double v = Store<S>::ld(pop + slot[r]);
          mom[0] += v * D::cx(r);
          mom[1] += v * D::cy(r);
          mom[2] += v * D::cz(r);
        }
        const double tq[3] = {arm_n[1] * mom[2] - arm_n[2] * mom[1], arm_n[2] * mom[0] - arm_n[0] * mom[2],
                              arm_n[0] * mom[1] - arm_n[1] * mom[0]};
        atomic_add3(pv.PF + 3 * nw, mom);
        atomic_add3(pv.PT + 3 * nw, tq);
      }
    } else if (old >= 0) {
      const double mom[3] = {pv.rho0 * u_o[0], pv.rho0 * u_o[1], pv.rho0 * u_o[2]};
      const double tq[3] = {arm_o[1] * mom[2] - arm_o[2] * mom[1], arm_o[2] * mom[0] - arm_o[0] * mom[2],
                            arm_o[0] * mom[1] - arm_o[1] * mom[0]};
      const double mneg[3] = {-mom[0], -mom[1], -mom[2]}, tneg[3] = {-tq[0], -tq[1], -tq[2]};
      atomic_add3(pv.PF + 3 * old, mneg);
      atomic_add3(pv.PT + 3 * old, tneg);
      if (nw == FLUID) {
        // uncovered: new fluid at n^eq(rho_bar, u_rigid), stored shifted
        const double uu = u_o[0] * u_o[0] + u_o[1] * u_o[1] + u_o[2] * u_o[2];
        for (int r = 0; r < Q; ++r) {
          const double cu = D::cx(r) * u_o[0] + D::cy(r) * u_o[1] + D::cz(r) * u_o[2];
          const double w = D::m(r) / 36.0;
          const double feq = pv.rho0 * w * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu + 4.5 * cu * cu * cu - 4.5 * uu * cu);
          Store<S>::st(pop + slot[r], (float)feq);
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

// owners >= 0 become resting fluid (first particles_set), layout of parity par
template <class S>
__global__ void k_clear_cells(LatticeView lv, int par) {
  const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= lv.N) return;
  if (lv.owner[n] < 0) return;
  lv.owner[n] = FLUID;
  const int x = n % lv.nx, y = (n / lv.nx) % lv.ny, z = n / ((unsigned)lv.nx * lv.ny);
  unsigned slot[Q];
  node_slots<S>(lv, par, x, y, z, slot);
  S *pop = reinterpret_cast<S *>(lv.pop);
  for (int r = 0; r < Q; ++r) Store<S>::st(pop + slot[r], 0.0f);
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

void launch_forces(const LatticeView &lv, const PartView &pv, const CellListView &cl, const WallRows &wr,
                   cudaStream_t st, int64_t *nl) {
  if (pv.n == 0) return;
  k_forces<<<nblk((unsigned)pv.n * 32, 128), 128, 0, st>>>(lv, pv, cl, wr);
  *nl += 1;
}

void launch_integrate_claim(const LatticeView &lv, const PartView &pv, int *claim, const ChangeList &chg, int mode,
                            cudaStream_t st, int64_t *nl) {
  if (pv.n == 0) return;
  k_integrate_claim<<<pv.n, 256, 0, st>>>(lv, pv, claim, chg, mode);
  *nl += 1;
}

void launch_resolve_fill(int dtype, const LatticeView &lv, const PartView &pv, int *claim, const ChangeList &chg,
                         const LinkList &ll, int par_next, int impulses, cudaStream_t st, int64_t *nl) {
  if (pv.n == 0) return;
  if (dtype == 0) k_resolve_fill<float><<<pv.n, 256, 0, st>>>(lv, pv, claim, chg, ll, par_next, impulses);
  else if (dtype == 1) k_resolve_fill<__nv_bfloat16><<<pv.n, 256, 0, st>>>(lv, pv, claim, chg, ll, par_next, impulses);
  else k_resolve_fill<__half><<<pv.n, 256, 0, st>>>(lv, pv, claim, chg, ll, par_next, impulses);
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
