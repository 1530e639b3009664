// bl_internal.cuh -- device-side definitions shared by the library's kernels.
//
// The method is the coupled step of arXiv:1005.2594 (Sec. II, III); this file
// holds only lattice constants, the views passed to kernels and small device
// helpers.  Nothing here is shared with the CPU oracle.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace bl {

constexpr int Q = 19;
constexpr int FLUID = -1;
constexpr int NWALL = 8;

// D3Q19 in the interface order (Sec. II): rest, 6 axis vectors, 12 diagonals,
// each followed by its opposite.  m = 36 alpha (alpha = 1/3, 1/18, 1/36).
struct D3Q19 {
  static __host__ __device__ constexpr int cx(int r) {
    return (r == 1 || r == 7 || r == 9 || r == 11 || r == 13) ? 1 : ((r == 2 || r == 8 || r == 10 || r == 12 || r == 14) ? -1 : 0);
  }
  static __host__ __device__ constexpr int cy(int r) {
    return (r == 3 || r == 7 || r == 10 || r == 15 || r == 17) ? 1 : ((r == 4 || r == 8 || r == 9 || r == 16 || r == 18) ? -1 : 0);
  }
  static __host__ __device__ constexpr int cz(int r) {
    return (r == 5 || r == 11 || r == 14 || r == 15 || r == 18) ? 1 : ((r == 6 || r == 12 || r == 13 || r == 16 || r == 17) ? -1 : 0);
  }
  static __host__ __device__ constexpr int opp(int r) { return r == 0 ? 0 : ((r & 1) ? r + 1 : r - 1); }
  static __host__ __device__ constexpr int m(int r) { return r == 0 ? 12 : (r <= 6 ? 2 : 1); }
};

// compile-time loop: f(std::integral_constant<int, I>) for I in [B, E)
template <int B, int E, class F>
__device__ __forceinline__ void sfor(F &&f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    sfor<B + 1, E>(f);
  }
}

// storage of the shifted populations f~ = f - alpha rho_bar
template <class S>
struct Store;
template <>
struct Store<float> {
  static __device__ __forceinline__ float ld(const float *p) { return *p; }
  static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};
template <>
struct Store<__nv_bfloat16> {
  static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};
// FP16 stores f~ scaled by 2^10 so that small deviations stay in the normal range
template <>
struct Store<__half> {
  static __device__ __forceinline__ float ld(const __half *p) { return __half2float(*p) * (1.0f / 1024.0f); }
  static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v * 1024.0f); }
};

// division by a lattice extent through a multiply-high: with
// m = floor((2^64 - 1) / d) + 1, floor(n / d) is the high 64 bits of n m for
// every 32-bit n and 2 <= d < 2^32 (m = floor(2^64 / d) + 1, or 2^64 / d when
// d divides 2^64; the error of n m / 2^64 against n / d is below n / 2^64 <
// 2^-32 <= 1 / d, and frac(n / d) <= 1 - 1 / d); d = 1 is passed through
struct FastDiv {
  unsigned long long m;
  unsigned d;
};
inline FastDiv make_fastdiv(unsigned d) {
  FastDiv f;
  f.d = d;
  f.m = d > 1u ? ~0ull / d + 1ull : 0ull;
  return f;
}
__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv &f) {
  return f.d == 1u ? n : (unsigned)__umul64hi((unsigned long long)n, f.m);
}

struct LatticeView {
  int nx, ny, nz;
  int per[3];
  unsigned N;  // nodes; 19 N < 2^32 is checked on the host
  FastDiv dnx, dnxy;  // division by nx and by nx ny (node index -> coordinates)
  float wall_vel[NWALL][3];
  float omega;  // 1 / tau
  float rho0;
  float g[3];
  int has_force;
  int sweep;  // sweep variant (0 one node per thread, 1 / 2 FP32 pipeline over 4 / 8 planes,
             // 3 / 4 bulk-copy pipeline over 8 / 4 planes, 5 persistent bulk-copy rows)
  int rows_grid[8];  // grid of the persistent row sweep per (parity, force, tau = 1)
  void *pop;       // 19 x N storage elements, slot r of node n at r * N + n
  int32_t *owner;  // N
  uint32_t *nbm;   // N neighbour words of the current owner map (NB_* bits), written by the geometry pass
  uint32_t *nbc;   // N neighbour-cell words (NBC_*), written with the neighbour words
  // Cell links of the sweep.  A fluid node next to a cell writes one link
  // record per cell into that cell's bucket, for the link-momentum sums.
  // The moving-boundary term C of its bounced populations needs the cell's
  // velocity of the half step, solved after the sweep: after the solve, the
  // node's record of its first cell becomes pu[n] = (rho (V + W x d), mask of
  // the bounced directions as the bits of .w), which the next sweep reads
  // with the populations and adds as C = -(m_r / 6) c_r . u; the links to a
  // second or third cell of one node get C in place right after the solve.
  float4 *pu;              // N
  float4 *rec;             // ncells x rec_cap records of 2 float4
  int *rec_count;          // ncells
  int rec_cap;
  int *status;
  // Lees-Edwards shear (null when off): the sweep leaves (drho, u) of the
  // nodes at x = 0 (first ny nz) and x = nx - 1 (next ny nz), y + ny z
  float4 *le_mom;
};

// Lees-Edwards shear across the plane between x = nx - 1 and x = 0 (Sec. IV,
// reading Q25): the image above moves with velocity offset U along z and is
// displaced by U t
struct LeView {
  double U;
  double *D;     // offset of the pass in flight: written by the gather, read by the scatter
  long long *t;  // steps since the shear was set
  double *P;     // z-momentum moved along +x across the plane, summed over the steps
  long long *n;  // steps summed
  float *T;      // 2 x 5 x ny nz crossing populations of the two planes, shifted to the other frame
};

// A link record (two float4): node n (bits of .x), direction mask (bits of
// .y: bit r = the neighbour n + c_r belongs to the cell; bit 31 marks the
// links of a node's second or third cell, whose C is given in place right
// after the solve), the density deviation drho = rho - rho_bar (.z), then
// at tau = 1 the node's velocity u (.w, second .x, .y), uu (second .z) and
// u . F (second .w), from which the link sums rebuild the bounced
// populations; at any other tau the sum over the mask of 2 f~*_r c_r (.w,
// second .x, .y).
constexpr uint32_t REC_DIRECT = 1u << 31;

// neighbour word of a node: bit 0 the node is fluid; bit r (1..18) the
// neighbour x + c_r is solid; NB_WALL some solid neighbour is a wall node;
// NB_CELL some solid neighbour is a cell node.  For a cell node (bit 0
// clear) bit r marks a contact link: the neighbour x + c_r is a wall node or
// a node of another cell.  Zero for wall nodes.
constexpr uint32_t NB_FLUID = 1u;
constexpr uint32_t NB_SOLID = 0x7FFFEu;
constexpr uint32_t NB_WALL = 1u << 19;
constexpr uint32_t NB_CELL = 1u << 20;
// neighbour-cell word of a fluid node next to a cell: the index of the cell
// owning its first solid neighbour in direction order (low bits), and
// NBC_MIXED when not every solid neighbour belongs to that cell (a wall or a
// second cell among them: the sweep then reads the neighbours' owners)
constexpr uint32_t NBC_MIXED = 1u << 31;
constexpr uint32_t NBC_CELL = 0x7FFFFFFFu;

// momentum given to each wall id by its bounce-back links: variable part in
// FP64, constant part 2 alpha_r rho_bar c_r as exact integer sums of m_r c_r
struct WallAcc {
  double *F;     // 8 x 3
  long long *K;  // 8 x 3
};

// Cells.  Their bounce links come from the sweep's link records
// (LatticeView::rec); contact links enter as exact integer sums cK, cIT.
struct PartView {
  int n;
  double *X, *q, *V, *L, *Om;
  double *o;         // exact FP64 symmetry axis of the current q, n x 3
  float *oprev;      // n x 3 axis before the last move (FP32): the claims' old ellipsoid
  float4 *kin;       // kinematics of the current step, 3 float4 per cell:
                     //   (f.x, f.y, f.z, Xi.x), (V, Xi.y), (W, Xi.z); X = Xi + f, Xi = rint(X)
  float4 *kin_next;  // kinematics written for the next step
  int *rec_last;     // n: records of the last sweep (for the link read-out)
  int *cK, *cIT;     // n x 3 each: contact links, sum m_r c_r and sum m_r dI x c_r
  unsigned long long *touched;  // n x touched_cap nodes claimed or left in one re-discretisation (pack_xyzr)
  double *lsum;      // n x 27 link sums of one step: F, T (variable part), Zff 6, Zft 9, Ztt 6
  int *lsum_i;       // n x 6 integer link sums: K, IT
  float *vw;         // n x 6 velocities of the half step the bounced populations are given
  int *touched_count;
  int touched_cap;
  double *Fpot, *Tpot;                 // potentials of the current step
  double *PF, *PT;                     // pending fill/drain impulses
  double *Flink, *Tlink, *Ftot, *Ttot; // read-out of the last step
  int *box;                            // n x 6 inclusive node box lo[3], hi[3]
  double *stage;                       // n x 13 staged state for particles_set
  int *status;                         // device status word (ST_* bits)
  double m, Iperp, Ipar, rho0;
  double g[3];
  int bfc, move;
  double le_dr;  // Lees-Edwards: reflect a cell within le_dr of the sheared plane (0: no shear)
  double inv_rpar2, inv_rperp2, R_par, R_perp;
  float sig_par, sig_perp, eps, eps_w, mu, nu, chi_prime, r_cut;
  float chi, sigbar, sigbar_w, chi_w, sigw_max;
  double chi_d, sigbar_d, sigbar_w_d, chi_w_d;  // the same in FP64 (contact geometry)
};

struct CellListView {
  int nb[3];
  int nbins;
  int *bin_of, *count, *start, *cursor, *ids;
};

// surface wall nodes (Sec. III: walls linked to the lumen) as one bit per
// node, rows of nxw 32-bit words along x
struct SurfBits {
  uint32_t *bits;  // ny nz nxw words, or null when there is no surface wall node
  int nxw;
  uint32_t *rows;  // one bit per lattice row (y, z): the row holds a surface wall node
};

// close pairs of the learned correction: pairs (i, j), their features
// (14 floats) and the network's outputs (6 floats)
struct PairBuf {
  int2 *pairs;
  float *feat, *out;
  int *count;
  int cap;
};

struct ChangeList {
  int *count;
  int32_t *items;  // triples (node, old, new)
  int cap;
};

// ---------------------------------------------------------------------------
// launchers (each adds the number of kernels it launched to *nl where given)

void launch_lb_step(int dtype, const LatticeView &lv, int par, const WallAcc &wa, int *status, cudaStream_t st);
// the persistent row sweep's grid per instantiation (LatticeView::rows_grid)
void lb_rows_grids(int dtype, int out[8]);
void launch_fields(int dtype, const LatticeView &lv, int par, double *rho, double *u, int32_t *owner,
                   cudaStream_t st);
void launch_pop_io(int dtype, const LatticeView &lv, int par, double *buf, int to_storage, cudaStream_t st);
void launch_init(int dtype, const LatticeView &lv, cudaStream_t st);
void launch_fill_int(int *a, unsigned n, int v, cudaStream_t st);
void launch_apply_wall_mask(const LatticeView &lv, const uint8_t *mask, cudaStream_t st);
void launch_surface_bits(const LatticeView &lv, const SurfBits &sb, int *count, cudaStream_t st);
void launch_surface_rows(const LatticeView &lv, const SurfBits &sb, cudaStream_t st);
unsigned links_blocks(const LatticeView &lv);
void launch_links(const LatticeView &lv, int contact, int pass, int *block_count, const int *block_off, int32_t *out,
                  long long cap, cudaStream_t st);
void launch_cell_list(const LatticeView &lv, const PartView &pv, const CellListView &cl, cudaStream_t st, int64_t *nl);
void launch_forces(const LatticeView &lv, const PartView &pv, const CellListView &cl, const SurfBits &sb,
                   cudaStream_t st, int64_t *nl);
// link sums from the sweep's records and the implicit solve + leap-frog;
// then the pending C of the records (independent of the claims, which need
// only the solve)
void launch_sums_solve(int dtype, const LatticeView &lv, const PartView &pv, int par, cudaStream_t st, int64_t *nl);
void launch_link_pending(int dtype, const LatticeView &lv, const PartView &pv, int par, cudaStream_t st,
                         int64_t *nl);
void launch_set_state(const LatticeView &lv, const PartView &pv, int mode, cudaStream_t st, int64_t *nl);
void launch_claims(const LatticeView &lv, const PartView &pv, int *claim, const ChangeList &chg, int mode,
                   cudaStream_t st, int64_t *nl);
void launch_geometry(const LatticeView &lv, const PartView &pv, cudaStream_t st, int64_t *nl);
// the geometry after a step's resolve, in two independent parts (together
// the same result as launch_geometry): neighbour words around the changed
// nodes (after resolve); contact sums cell by cell from the current owner
// map and kinematics (at the start of the next step)
void launch_nbm_update(const LatticeView &lv, const PartView &pv, const ChangeList &chg, cudaStream_t st,
                       int64_t *nl);
void launch_contacts(const LatticeView &lv, const PartView &pv, cudaStream_t st, int64_t *nl);
// the pending C of the last step into the stored populations (layout par),
// before read-outs and state changes between steps
void launch_flush_pending(int dtype, const LatticeView &lv, int par, cudaStream_t st, int64_t *nl);
void launch_resolve_fill(int dtype, const LatticeView &lv, const PartView &pv, const CellListView &cl, int *claim,
                         const ChangeList &chg, int par_next, int impulses, cudaStream_t st, int64_t *nl);
void launch_clear_cells(int dtype, const LatticeView &lv, int par, cudaStream_t st, int64_t *nl);

void launch_pair_features(const LatticeView &lv, const PartView &pv, const int2 *pairs, int n, float *out,
                          cudaStream_t st);
void launch_mlp_correction(const LatticeView &lv, const PartView &pv, const CellListView &cl, const PairBuf &pb,
                           float gap_lo, float gap_cut, float speed_lo, float speed_hi, const void *mlp,
                           cudaStream_t st, int64_t *nl);
// forward pass of a bl_mlp over *count rows of x (at most cap), raw units
void launch_mlp_forward_dev(const void *mlp, const float *x, const int *count, int cap, float *y, cudaStream_t st);
// the Lees-Edwards passes after a sweep of parity par
void launch_lees_edwards(int dtype, const LatticeView &lv, const LeView &le, int par, cudaStream_t st, int64_t *nl);

// bit flags of the device status word
constexpr int ST_UNSTABLE = 1;
constexpr int ST_OVERFLOW = 2;
constexpr int ST_BARRIER = 4;  // a bounded wait on an mbarrier gave up
constexpr int ST_LEPLANE = 8;  // a node beside the Lees-Edwards plane is not fluid

// ---------------------------------------------------------------------------
// exact FP64 geometry (no contraction), matching the operation order of the
// plain reference so that inside decisions agree bit for bit

__device__ __forceinline__ void axis_exact(const double *q, double *o) {
  o[0] = __dmul_rn(2.0, __dadd_rn(__dmul_rn(q[1], q[3]), __dmul_rn(q[0], q[2])));
  o[1] = __dmul_rn(2.0, __dsub_rn(__dmul_rn(q[2], q[3]), __dmul_rn(q[0], q[1])));
  o[2] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(__dmul_rn(q[1], q[1]), __dmul_rn(q[2], q[2]))));
}

__device__ __forceinline__ double min_image_exact(double d, int n, int per) {
  if (!per) return d;
  double half = __dmul_rn(0.5, (double)n);
  if (d > half) return __dsub_rn(d, (double)n);
  if (d < -half) return __dadd_rn(d, (double)n);
  return d;
}

__device__ __forceinline__ bool inside_exact(int x, int y, int z, const double *X, const double *o,
                                             double inv_rpar2, double inv_rperp2, const LatticeView &lv) {
  double d0 = min_image_exact(__dsub_rn((double)x, X[0]), lv.nx, lv.per[0]);
  double d1 = min_image_exact(__dsub_rn((double)y, X[1]), lv.ny, lv.per[1]);
  double d2 = min_image_exact(__dsub_rn((double)z, X[2]), lv.nz, lv.per[2]);
  double dpar = __dadd_rn(__dadd_rn(__dmul_rn(d0, o[0]), __dmul_rn(d1, o[1])), __dmul_rn(d2, o[2]));
  double dd = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
  double pp = __dmul_rn(dpar, dpar);
  double s = __dadd_rn(__dmul_rn(pp, inv_rpar2), __dmul_rn(__dsub_rn(dd, pp), inv_rperp2));
  return s <= 1.0;
}

// integer minimum image of a lattice displacement
__device__ __forceinline__ int imin_image(int d, int n, int per) {
  if (!per) return d;
  if (2 * d > n) return d - n;
  if (2 * d < -n) return d + n;
  return d;
}

// periodic wrap for coordinates at most a few periods out (no division)
__device__ __forceinline__ int wrapi(int v, int n) {
  while (v < 0) v += n;
  while (v >= n) v -= n;
  return v;
}

// packed node coordinates of the per-cell lists: r | x << 5 | y << 25 | z << 45
__host__ __device__ __forceinline__ unsigned long long pack_xyzr(int x, int y, int z, int r) {
  return (unsigned long long)r | ((unsigned long long)x << 5) | ((unsigned long long)y << 25) |
         ((unsigned long long)z << 45);
}
__device__ __forceinline__ void unpack_xyzr(unsigned long long e, int xyz[3], int &r) {
  r = (int)(e & 31ull);
  xyz[0] = (int)((e >> 5) & 0xFFFFFull);
  xyz[1] = (int)((e >> 25) & 0xFFFFFull);
  xyz[2] = (int)(e >> 45);
}

// direction masks of the lattice (bit r), for the record sums by popcount
template <class P>
__host__ __device__ constexpr uint32_t dir_mask(P pred) {
  uint32_t m = 0;
  for (int r = 1; r < Q; ++r)
    if (pred(r)) m |= 1u << r;
  return m;
}
using D3 = D3Q19;
constexpr int cxyz(int r, int a) { return a == 0 ? D3::cx(r) : (a == 1 ? D3::cy(r) : D3::cz(r)); }
template <int A, int SGN>
struct AxisDirs {  // axis vectors along A with sign SGN (m = 2)
  static constexpr uint32_t v = dir_mask([](int r) { return r <= 6 && cxyz(r, A) == SGN; });
};
template <int A, int SGN>
struct DiagDirs {  // diagonal vectors with c_A = SGN (m = 1)
  static constexpr uint32_t v = dir_mask([](int r) { return r > 6 && cxyz(r, A) == SGN; });
};
template <int A, int B, int SGN>
struct PairDirs {  // diagonal vectors with c_A c_B = SGN
  static constexpr uint32_t v = dir_mask([](int r) { return r > 6 && cxyz(r, A) * cxyz(r, B) == SGN; });
};

__device__ __forceinline__ int popm(uint32_t m, uint32_t sel) { return __popc(m & sel); }

// the components of c_r for a direction r known only at run time: c + 1
// packed two bits per direction in a 64-bit constant
template <int A>
__host__ __device__ constexpr unsigned long long packed_dirs() {
  unsigned long long v = 0;
  for (int r = 0; r < Q; ++r) v |= (unsigned long long)(cxyz(r, A) + 1) << (2 * r);
  return v;
}
template <int A>
__device__ __forceinline__ int rt_c(int r) {
  return (int)((packed_dirs<A>() >> (2 * r)) & 3ull) - 1;
}
__device__ __forceinline__ int rt_m(int r) { return r == 0 ? 12 : (r <= 6 ? 2 : 1); }
__device__ __forceinline__ int rt_opp(int r) { return r == 0 ? 0 : ((r & 1) ? r + 1 : r - 1); }

// node index -> coordinates
__device__ __forceinline__ void node_xyz(const LatticeView &lv, unsigned n, int xyz[3]) {
  const unsigned z = fdiv(n, lv.dnxy), rem = n - z * lv.dnxy.d, y = fdiv(rem, lv.dnx);
  xyz[0] = (int)(rem - y * lv.dnx.d);
  xyz[1] = (int)y;
  xyz[2] = (int)z;
}

// sums over the directions of a mask (bit r) by popcount: component A of
// K = sum m_r c_r, and the entries A A and A B of M = sum m_r c_r c_r^T
template <int A>
__device__ __forceinline__ int mask_K(uint32_t m) {
  return 2 * (popm(m, AxisDirs<A, 1>::v) - popm(m, AxisDirs<A, -1>::v)) + popm(m, DiagDirs<A, 1>::v) -
         popm(m, DiagDirs<A, -1>::v);
}
template <int A>
__device__ __forceinline__ int mask_Maa(uint32_t m) {
  return 2 * popm(m, AxisDirs<A, 1>::v | AxisDirs<A, -1>::v) + popm(m, DiagDirs<A, 1>::v | DiagDirs<A, -1>::v);
}
template <int A, int B>
__device__ __forceinline__ int mask_Mab(uint32_t m) {
  return popm(m, PairDirs<A, B, 1>::v) - popm(m, PairDirs<A, B, -1>::v);
}

// post-collision shifted population at tau = 1: the third-order equilibrium
// w (drho + rho t), t = 4.5 cu^2 - 1.5 uu + cu (3 - 4.5 uu + 4.5 cu^2), with
// rho t taken as rho_bar t + drho t (exact for small drho in FP32), plus the
// Guo source src_w w (3 (cF - uF) + 9 cu cF) when a force acts; the sweep and
// the link sums evaluate this same function, so the bounced populations the
// fluid keeps and those the cell's momentum counts agree
__device__ __forceinline__ float post_tau1(float w, float drho, float rho0, float cu, float uu, bool force, float cF,
                                           float uF, float src_w) {
  const float q = 4.5f * cu * cu;
  const float t = (q - 1.5f * uu) + cu * ((3.0f - 4.5f * uu) + q);
  float fs = w * (drho + fmaf(drho, t, rho0 * t));
  if (force) fs += src_w * w * (3.0f * (cF - uF) + 9.0f * cu * cF);
  return fs;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace bl
