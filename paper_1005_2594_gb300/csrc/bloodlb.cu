// bloodlb.cu -- host side of the C ABI declared in include/bloodlb.h.
//
// One context owns one lattice and its cells on one CUDA stream.  A time step
// (arXiv:1005.2594, Sec. II and III) is enqueued as five kernel groups (the
// groups of the timing read-out):
//   0  fused collide / stream / bounce-back / wall momentum / pending
//      moving-boundary term / cell-link records (the sweep)
//   1  cell list (count, scan, scatter, per-bin sort)
//   2  pair and wall potentials (+ the learned correction)
//   3  link sums, implicit solve + leap-frog, claims, pending terms
//   4  contact sums, resolve + fill/drain, neighbour words
// Groups 1-2 and the contact sums run on two side streams beside the sweep,
// the claims beside the pending terms.  The host never waits inside
// bl_step; device failures are raised into a status word that bl_sync reads.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <utility>
#include <vector>

#include "../../include/bloodlb.h"
#include "bl_internal.cuh"

using namespace bl;

namespace {
constexpr int NGROUPS = 5;
constexpr int MAX_TIMED = 1 << 16;
}  // namespace

struct bl_ctx {
  bl_lb_params lp;
  bl_particle_params pp;
  cudaStream_t stream;  // the caller's stream: every call is ordered on it
  // the cell list and the potentials of a step run on a second stream, the
  // contact sums on a third, overlapped with the lattice sweep (they touch
  // disjoint data); the claims run on the second beside the pending terms
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;     // cell list and potentials beside the sweep
  cudaEvent_t ev_fork2, ev_join2;   // claims beside the pending terms
  cudaStream_t side2;
  cudaEvent_t ev_join3;             // contact sums beside the sweep (second side stream)
  // repeated steps replay a CUDA graph of two steps (even + odd parity), a
  // lone step a one-step graph, on an internal stream forked from and joined
  // to the caller's stream
  cudaStream_t gstream;
  cudaGraphExec_t gexec;
  cudaGraphExec_t g1exec[2];  // one step from parity 0 / 1 (for odd step counts)
  const void *g1kin[2];
  int64_t g1_launches[2];
  int g_parity;
  const void *g_kin;
  int64_t g_launches;
  int epoch;  // counts graph invalidations (cell arrays moved, walls or sweep variant changed)
  // learned near-contact correction (bl_mlp_attach_range): the model, the
  // gap and relative-speed window it is used in, the close-pair buffers
  // (32 pairs per cell)
  const void *mlp;
  float gap_lo, gap_cut, speed_lo, speed_hi;
  PairBuf pb;
  int dtype;
  int parity;  // layout of the current populations (next step's parity)
  LatticeView lv;
  int *claim;
  int *status;
  int sticky;
  char err[256];
  int64_t launches;
  // walls
  WallAcc wacc;
  SurfBits sbits;
  // cells
  int np;
  PartView pv;
  CellListView cl;
  ChangeList chg;
  // scratch for read-outs
  double *scratch;
  size_t scratch_bytes;
  // timing
  // Lees-Edwards shear (bl_lees_edwards_set): its passes run after every
  // sweep; masked: a wall mask was set (the shear needs fluid planes)
  LeView le;
  int le_on;
  double le_dr_req;  // reflection distance asked for (<= 0: the default)
  int masked;
  int timing;
  int sweep_fixed;  // the sweep variant was set (bl_sweep_variant, bl_autotune), not chosen here
  std::vector<cudaEvent_t> ev;  // pairs
  std::vector<int> ev_group;
  int ev_used;
  double t_ms[NGROUPS];
  int64_t t_cnt[NGROUPS];
};

static void drop_graph(bl_ctx *c);
static int read_status(bl_ctx *c);
static void fill_particle_constants(bl_ctx *c);

static int fail(bl_ctx *c, int code, const char *fmt, ...) {
  if (c && c->sticky == BL_OK) {
    c->sticky = code;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define CU(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(c, e_ == cudaErrorMemoryAllocation ? BL_ENOMEM : BL_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                         \
  } while (0)

static int check_launch(bl_ctx *c, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, BL_ECUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
  return BL_OK;
}

static size_t elem_size(int dtype) { return dtype == BL_STORE_F32 ? 4 : 2; }

// the sweep variant of a context that was given none.  With cells, one node
// per thread: the boundary work of a suspension falls unevenly on the warps,
// and hiding its latency by occupancy beats a block-wide copy pipeline whose
// barriers make every warp wait for the slowest.  Without cells, the
// bulk-copy pipeline over 8 planes where rows are 16-byte aligned, else the
// FP32 per-thread copy pipeline or one node per thread.
static int auto_sweep(const bl_ctx *c) {
  if (c->np > 0) return 0;
  if (c->lv.nx % (c->dtype == BL_STORE_F32 ? 4 : 8) == 0) return 3;
  return c->dtype == BL_STORE_F32 ? 1 : 0;
}

static int ensure_scratch(bl_ctx *c, size_t bytes) {
  if (c->scratch_bytes >= bytes) return BL_OK;
  if (c->scratch) cudaFree(c->scratch);
  c->scratch = nullptr;
  c->scratch_bytes = 0;
  CU(cudaMalloc(&c->scratch, bytes));
  c->scratch_bytes = bytes;
  return BL_OK;
}

// ---------------------------------------------------------------------------
// timing

static void group_begin(bl_ctx *c, int g, int *slot, cudaStream_t st) {
  *slot = -1;
  if (!c->timing || c->ev_used >= MAX_TIMED) return;
  const int s = c->ev_used++;
  if ((int)c->ev.size() < 2 * (s + 1)) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return;
    c->ev.push_back(a);
    c->ev.push_back(b);
    c->ev_group.push_back(g);
  }
  c->ev_group[s] = g;
  cudaEventRecord(c->ev[2 * s], st);
  *slot = s;
}

static void group_end(bl_ctx *c, int slot, cudaStream_t st) {
  if (slot >= 0) cudaEventRecord(c->ev[2 * slot + 1], st);
}

static int harvest_timing(bl_ctx *c) {
  if (c->ev_used == 0) return BL_OK;
  CU(cudaStreamSynchronize(c->stream));
  for (int s = 0; s < c->ev_used; ++s) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[2 * s], c->ev[2 * s + 1]) == cudaSuccess) {
      c->t_ms[c->ev_group[s]] += ms;
      c->t_cnt[c->ev_group[s]] += 1;
    }
  }
  c->ev_used = 0;
  return BL_OK;
}

// ---------------------------------------------------------------------------
// surface wall nodes (Sec. III: wall spheres at wall nodes linked to the lumen)

static int build_surface_bits(bl_ctx *c) {
  c->sbits.nxw = (c->lv.nx + 31) / 32;
  const size_t words = (size_t)c->sbits.nxw * c->lv.ny * c->lv.nz;
  uint32_t *bits = c->sbits.bits;
  if (!bits) CU(cudaMalloc(&bits, sizeof(uint32_t) * words));
  const size_t rwords = ((size_t)c->lv.ny * c->lv.nz + 31) / 32;
  uint32_t *rows = c->sbits.rows;
  if (!rows) CU(cudaMalloc(&rows, sizeof(uint32_t) * rwords));
  int *cnt = nullptr;
  CU(cudaMalloc(&cnt, sizeof(int)));
  CU(cudaMemsetAsync(cnt, 0, sizeof(int), c->stream));
  SurfBits sb = {bits, c->sbits.nxw, rows};
  launch_surface_bits(c->lv, sb, cnt, c->stream);
  CU(cudaMemsetAsync(rows, 0, sizeof(uint32_t) * rwords, c->stream));
  launch_surface_rows(c->lv, sb, c->stream);
  c->launches += 2;
  int h = 0;
  CU(cudaMemcpyAsync(&h, cnt, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  cudaFree(cnt);
  if (check_launch(c, "surface bits")) return c->sticky;
  if (h == 0) {
    cudaFree(bits);  // no walls: the wall potential is skipped
    cudaFree(rows);
    bits = nullptr;
    rows = nullptr;
  }
  c->sbits.bits = bits;
  c->sbits.rows = rows;
  return BL_OK;
}

// The steps leave the moving-boundary term C of their last bounces off cells
// pending (the next sweep adds it as it reads the populations): before the
// populations are read out or the cells are set anew, it is given to the
// stored populations here.
static int flush_pending(bl_ctx *c) {
  if (c->np == 0) return BL_OK;  // nothing pends without cells (a removal flushes first)
  launch_flush_pending(c->dtype, c->lv, c->parity, c->stream, &c->launches);
  return check_launch(c, "pending moving-boundary terms");
}

// ---------------------------------------------------------------------------
// C ABI

extern "C" int bl_lb_init(bl_ctx **out, const bl_lb_params *p, void *cuda_stream) {
  if (!out) return BL_EINVAL;
  *out = nullptr;
  if (!p) return BL_EINVAL;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || !(p->tau > 0.5) || !(p->rho0 > 0.0) || p->store_dtype < 0 ||
      p->store_dtype > 2)
    return BL_EINVAL;
  const unsigned long long N = (unsigned long long)p->nx * p->ny * p->nz;
  // 19 N slots index with 32 bits; per-cell lists pack x, y in 20 bits, z in 19
  if (N * bl::Q >= (1ull << 32) || p->nx >= (1 << 20) || p->ny >= (1 << 20) || p->nz >= (1 << 19)) return BL_EINVAL;
  for (int k = 0; k < 3; ++k) {
    const int n = k == 0 ? p->nx : (k == 1 ? p->ny : p->nz);
    if (!p->periodic[k] && n < 3) return BL_EINVAL;  // two wall layers and fluid between
  }
  bl_ctx *c = new bl_ctx();
  memset(c->err, 0, sizeof(c->err));
  c->lp = *p;
  c->stream = (cudaStream_t)cuda_stream;
  c->dtype = p->store_dtype;
  c->parity = 0;
  c->sticky = BL_OK;
  LatticeView &lv = c->lv;
  lv.nx = p->nx;
  lv.ny = p->ny;
  lv.nz = p->nz;
  for (int k = 0; k < 3; ++k) lv.per[k] = p->periodic[k] ? 1 : 0;
  lv.N = (unsigned)N;
  lv.dnx = bl::make_fastdiv((unsigned)p->nx);
  lv.dnxy = bl::make_fastdiv((unsigned)p->nx * (unsigned)p->ny);
  for (int w = 0; w < bl::NWALL; ++w)
    for (int k = 0; k < 3; ++k) lv.wall_vel[w][k] = (float)p->wall_vel[w][k];
  lv.omega = (float)(1.0 / p->tau);
  lv.rho0 = (float)p->rho0;
  lv.has_force = 0;
  // (no cells yet: the bulk-copy pipeline over 8 planes where rows are
  // 16-byte aligned, nx a multiple of 4 in FP32, of 8 in BF16 / FP16; else
  // FP32 takes the pipeline over 4 planes and 16-bit storage one node per
  // thread; auto_sweep changes it when cells come)
  if (p->store_dtype == BL_STORE_F32) lv.sweep = p->nx % 4 == 0 ? 3 : 1;
  else lv.sweep = p->nx % 8 == 0 ? 3 : 0;
  bl::lb_rows_grids(p->store_dtype, lv.rows_grid);
  for (int k = 0; k < 3; ++k) {
    lv.g[k] = (float)p->g[k];
    if (p->g[k] != 0.0) lv.has_force = 1;
  }
  int rc = BL_OK;
  do {
    if (cudaMalloc(&lv.pop, elem_size(c->dtype) * N * bl::Q) != cudaSuccess) { rc = fail(c, BL_ENOMEM, "population field"); break; }
    if (cudaMalloc(&lv.owner, sizeof(int32_t) * N) != cudaSuccess) { rc = fail(c, BL_ENOMEM, "owner map"); break; }
    if (cudaMalloc(&c->claim, sizeof(int) * N) != cudaSuccess) { rc = fail(c, BL_ENOMEM, "claim map"); break; }
    if (cudaMalloc(&c->status, sizeof(int)) != cudaSuccess) { rc = fail(c, BL_ENOMEM, "status"); break; }
    // the side streams run the cell list, the potentials, the contact sums
    // and the claims beside the sweep and the pending C: at the highest
    // priority, so that their few blocks are not queued behind the sweep's
    // thousands (the step waits for them before the link sums)
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork2, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithPriority(&c->side2, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join3, cudaEventDisableTiming) != cudaSuccess) {
      rc = fail(c, BL_ECUDA, "streams");
      break;
    }
    if (cudaMalloc(&c->wacc.F, sizeof(double) * bl::NWALL * 3) != cudaSuccess) { rc = fail(c, BL_ENOMEM, "wall"); break; }
    if (cudaMalloc(&c->wacc.K, sizeof(long long) * bl::NWALL * 3) != cudaSuccess) { rc = fail(c, BL_ENOMEM, "wall"); break; }
    cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
    cudaMemsetAsync(c->wacc.F, 0, sizeof(double) * bl::NWALL * 3, c->stream);
    cudaMemsetAsync(c->wacc.K, 0, sizeof(long long) * bl::NWALL * 3, c->stream);
    launch_init(c->dtype, lv, c->stream);
    launch_fill_int(c->claim, lv.N, INT_MAX, c->stream);
    c->launches += 2;
    if ((rc = check_launch(c, "init")) != BL_OK) break;
    if (cudaMalloc(&lv.nbm, sizeof(uint32_t) * N) != cudaSuccess) { rc = fail(c, BL_ENOMEM, "neighbour words"); break; }
    if (cudaMalloc(&lv.nbc, sizeof(uint32_t) * N) != cudaSuccess) { rc = fail(c, BL_ENOMEM, "neighbour-cell words"); break; }
    if (cudaMalloc(&lv.pu, sizeof(float4) * N) != cudaSuccess) { rc = fail(c, BL_ENOMEM, "pending velocities"); break; }
    cudaMemsetAsync(lv.pu, 0, sizeof(float4) * N, c->stream);
    lv.status = c->status;
    launch_geometry(lv, c->pv, c->stream, &c->launches);
    if ((rc = check_launch(c, "geometry")) != BL_OK) break;
    if ((rc = build_surface_bits(c)) != BL_OK) break;
  } while (0);
  if (rc != BL_OK) {
    bl_destroy(c);
    return rc;
  }
  *out = c;
  return BL_OK;
}

extern "C" int bl_walls_set(bl_ctx *c, const uint8_t *mask) {
  if (!c || !mask) return BL_EINVAL;
  if (c->sticky) return c->sticky;
  if (c->np > 0) return fail(c, BL_ESTATE, "bl_walls_set after bl_particles_set");
  for (size_t i = 0; i < c->lv.N; ++i)
    if (mask[i] > bl::NWALL) return fail(c, BL_EINVAL, "wall mask value %d > 8 at node %zu", (int)mask[i], i);
  bool any = false;
  for (size_t i = 0; i < c->lv.N && !any; ++i) any = mask[i] != 0;
  if (any && c->le_on) return fail(c, BL_ESTATE, "bl_walls_set with a Lees-Edwards shear (its planes must hold fluid)");
  if (any) c->masked = 1;
  uint8_t *d = nullptr;
  CU(cudaMalloc(&d, c->lv.N));
  CU(cudaMemcpyAsync(d, mask, c->lv.N, cudaMemcpyHostToDevice, c->stream));
  drop_graph(c);
  launch_apply_wall_mask(c->lv, d, c->stream);
  c->launches++;
  launch_geometry(c->lv, c->pv, c->stream, &c->launches);
  int rc = check_launch(c, "wall mask");
  cudaStreamSynchronize(c->stream);
  cudaFree(d);
  if (rc) return rc;
  return build_surface_bits(c);
}

static void free_particles(bl_ctx *c) {
  PartView &pv = c->pv;
  void *ptrs[] = {pv.X, pv.q, pv.V, pv.L, pv.Om, pv.o, pv.oprev, pv.kin, pv.kin_next, pv.rec_last, pv.cK, pv.cIT,
                  pv.touched, pv.touched_count, pv.lsum, pv.lsum_i, pv.vw, pv.Fpot, pv.Tpot, pv.PF, pv.PT, pv.Flink, pv.Tlink, pv.Ftot,
                  pv.Ttot, pv.box, pv.stage, c->cl.bin_of, c->cl.count, c->cl.start, c->cl.cursor, c->cl.ids,
                  c->chg.count, c->chg.items, c->lv.rec, c->lv.rec_count};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  c->lv.rec = nullptr;
  c->lv.rec_count = nullptr;
  c->lv.rec_cap = 0;
  {
    void *pp[] = {c->pb.pairs, c->pb.feat, c->pb.out, c->pb.count};
    for (void *p : pp)
      if (p) cudaFree(p);
    c->pb = PairBuf{};
  }
  memset(&c->pv, 0, sizeof(c->pv));
  memset(&c->cl, 0, sizeof(c->cl));
  memset(&c->chg, 0, sizeof(c->chg));
  c->np = 0;
}

static int alloc_particles(bl_ctx *c, int n) {
  PartView &pv = c->pv;
  const size_t n3 = sizeof(double) * 3 * (size_t)n;
  double **d3[] = {&pv.X, &pv.V, &pv.L, &pv.Om, &pv.o, &pv.Fpot, &pv.Tpot, &pv.PF, &pv.PT,
                   &pv.Flink, &pv.Tlink, &pv.Ftot, &pv.Ttot};
  for (double **d : d3) {
    CU(cudaMalloc(d, n3));
    CU(cudaMemsetAsync(*d, 0, n3, c->stream));
  }
  CU(cudaMalloc(&pv.oprev, sizeof(float) * 3 * (size_t)n));
  CU(cudaMemsetAsync(pv.oprev, 0, sizeof(float) * 3 * (size_t)n, c->stream));
  CU(cudaMalloc(&pv.q, sizeof(double) * 4 * (size_t)n));
  CU(cudaMemsetAsync(pv.q, 0, sizeof(double) * 4 * (size_t)n, c->stream));
  CU(cudaMalloc(&pv.kin, sizeof(float4) * 3 * (size_t)n));
  CU(cudaMalloc(&pv.kin_next, sizeof(float4) * 3 * (size_t)n));
  CU(cudaMemsetAsync(pv.kin, 0, sizeof(float4) * 3 * (size_t)n, c->stream));
  CU(cudaMemsetAsync(pv.kin_next, 0, sizeof(float4) * 3 * (size_t)n, c->stream));
  CU(cudaMalloc(&pv.box, sizeof(int) * 6 * (size_t)n));
  CU(cudaMemsetAsync(pv.box, 0, sizeof(int) * 6 * (size_t)n, c->stream));
  CU(cudaMalloc(&pv.stage, sizeof(double) * 13 * (size_t)n));
  CU(cudaMalloc(&pv.lsum, sizeof(double) * 27 * (size_t)n));
  CU(cudaMemsetAsync(pv.lsum, 0, sizeof(double) * 27 * (size_t)n, c->stream));
  CU(cudaMalloc(&pv.lsum_i, sizeof(int) * 6 * (size_t)n));
  CU(cudaMemsetAsync(pv.lsum_i, 0, sizeof(int) * 6 * (size_t)n, c->stream));
  CU(cudaMalloc(&pv.vw, sizeof(float) * 6 * (size_t)n));
  CU(cudaMemsetAsync(pv.vw, 0, sizeof(float) * 6 * (size_t)n, c->stream));
  CU(cudaMalloc(&pv.cK, sizeof(int) * 3 * (size_t)n));
  CU(cudaMalloc(&pv.cIT, sizeof(int) * 3 * (size_t)n));
  CU(cudaMemsetAsync(pv.cK, 0, sizeof(int) * 3 * (size_t)n, c->stream));
  CU(cudaMemsetAsync(pv.cIT, 0, sizeof(int) * 3 * (size_t)n, c->stream));
  // per-cell lists: link records of the sweep (one per fluid node next to
  // the cell: at most the nodes within one node of its surface, fewer than
  // twice the area of a sphere of radius max(R) + 1) and nodes touched by
  // one re-discretisation (at most the box)
  const double rmax = fmax(c->pp.R_par, c->pp.R_perp);
  const double rec_cap = 2.0 * 4.0 * M_PI * (rmax + 1.0) * (rmax + 1.0) + 64.0;
  const double box = 2.0 * rmax + 4.0;
  const double t_cap = box * box * box;
  if (rec_cap * n > 2.0e9 || t_cap * n > 2.0e9 || n > 65535) return fail(c, BL_EINVAL, "cell lists too large");
  c->lv.rec_cap = (int)rec_cap;
  pv.touched_cap = (int)t_cap;
  CU(cudaMalloc(&c->lv.rec, sizeof(float4) * 2 * (size_t)c->lv.rec_cap * n));
  CU(cudaMalloc(&c->lv.rec_count, sizeof(int) * (size_t)n));
  CU(cudaMemsetAsync(c->lv.rec_count, 0, sizeof(int) * (size_t)n, c->stream));
  CU(cudaMalloc(&pv.rec_last, sizeof(int) * (size_t)n));
  CU(cudaMemsetAsync(pv.rec_last, 0, sizeof(int) * (size_t)n, c->stream));
  CU(cudaMalloc(&pv.touched, sizeof(unsigned long long) * (size_t)pv.touched_cap * n));
  CU(cudaMalloc(&pv.touched_count, sizeof(int) * (size_t)n));
  CU(cudaMemsetAsync(pv.touched_count, 0, sizeof(int) * (size_t)n, c->stream));
  // cell list bins: nb_k = max(1, floor(N_k / r_cut))
  const int dims[3] = {c->lv.nx, c->lv.ny, c->lv.nz};
  // bin counts in double, checked before any conversion to int
  double nbins_d = 1.0;
  for (int k = 0; k < 3; ++k) {
    const double nb = fmax(1.0, floor((double)dims[k] / c->pp.r_cut));
    if (!(nb <= (double)(1 << 26))) return fail(c, BL_EINVAL, "r_cut gives too many bins");
    c->cl.nb[k] = (int)nb;
    nbins_d *= nb;
  }
  if (!(nbins_d <= (double)(1 << 26))) return fail(c, BL_EINVAL, "r_cut gives too many bins");
  const long long nbins = (long long)nbins_d;
  c->cl.nbins = (int)nbins;
  CU(cudaMalloc(&c->cl.bin_of, sizeof(int) * (size_t)n));
  CU(cudaMalloc(&c->cl.count, sizeof(int) * (size_t)nbins));
  CU(cudaMalloc(&c->cl.cursor, sizeof(int) * (size_t)nbins));
  CU(cudaMalloc(&c->cl.start, sizeof(int) * (size_t)(nbins + 1)));
  CU(cudaMalloc(&c->cl.ids, sizeof(int) * (size_t)n));
  CU(cudaMemsetAsync(c->cl.count, 0, sizeof(int) * (size_t)nbins, c->stream));
  CU(cudaMemsetAsync(c->cl.cursor, 0, sizeof(int) * (size_t)nbins, c->stream));
  // diagnostic list of changed nodes (overflow only truncates the list)
  c->chg.cap = 64 * n + 4096;
  CU(cudaMalloc(&c->chg.count, sizeof(int)));
  CU(cudaMalloc(&c->chg.items, sizeof(int32_t) * 3 * (size_t)c->chg.cap));
  CU(cudaMemsetAsync(c->chg.count, 0, sizeof(int), c->stream));
  c->np = n;
  pv.n = n;
  return BL_OK;
}

static int alloc_pairbuf(bl_ctx *c) {
  if (c->pb.pairs || c->np == 0) return BL_OK;
  PairBuf &pb = c->pb;
  pb.cap = 32 * c->np;
  CU(cudaMalloc(&pb.pairs, sizeof(int2) * (size_t)pb.cap));
  CU(cudaMalloc(&pb.feat, sizeof(float) * 14 * (size_t)pb.cap));
  CU(cudaMalloc(&pb.out, sizeof(float) * 6 * (size_t)pb.cap));
  CU(cudaMalloc(&pb.count, sizeof(int)));
  CU(cudaMemsetAsync(pb.count, 0, sizeof(int), c->stream));
  return BL_OK;
}

static void fill_particle_constants(bl_ctx *c) {
  const bl_particle_params &pp = c->pp;
  PartView &pv = c->pv;
  const double m = pp.rho_p * (4.0 / 3.0) * M_PI * pp.R_perp * pp.R_perp * pp.R_par;
  pv.m = m;
  pv.Iperp = m * (pp.R_par * pp.R_par + pp.R_perp * pp.R_perp) / 5.0;
  pv.Ipar = 2.0 * m * pp.R_perp * pp.R_perp / 5.0;
  pv.rho0 = c->lp.rho0;
  for (int k = 0; k < 3; ++k) pv.g[k] = c->lp.g[k];
  pv.status = c->status;
  pv.bfc = c->lp.body_force_on_cells ? 1 : 0;
  pv.move = pp.move_particles;
  // Sec. IV's reflection distance sigma_perp, raised to max(R) + 1 so that no
  // cell covers a node beside the sheared plane (reading Q25)
  pv.le_dr = !c->le_on ? 0.0
                       : (c->le_dr_req > 0.0 ? c->le_dr_req
                                             : fmax(pp.sig_perp, fmax(pp.R_perp, pp.R_par) + 1.0));
  pv.inv_rpar2 = 1.0 / (pp.R_par * pp.R_par);
  pv.inv_rperp2 = 1.0 / (pp.R_perp * pp.R_perp);
  pv.R_par = pp.R_par;
  pv.R_perp = pp.R_perp;
  pv.sig_par = (float)pp.sig_par;
  pv.sig_perp = (float)pp.sig_perp;
  pv.eps = (float)pp.eps;
  pv.eps_w = (float)pp.eps_w;
  pv.mu = (float)pp.mu;
  pv.nu = (float)pp.nu;
  pv.chi_prime = (float)pp.chi_prime;
  pv.r_cut = (float)pp.r_cut;
  const double sp2 = pp.sig_par * pp.sig_par, sq2 = pp.sig_perp * pp.sig_perp, sw2 = pp.sig_w * pp.sig_w;
  pv.chi = (float)((sp2 - sq2) / (sp2 + sq2));
  pv.sigbar = (float)(2.0 * pp.sig_perp);
  pv.sigbar_w = (float)sqrt(sq2 + sw2);
  const double chi_w = (sp2 - sq2) / (sp2 + sw2);
  pv.chi_w = (float)chi_w;
  pv.chi_d = (sp2 - sq2) / (sp2 + sq2);
  pv.sigbar_d = 2.0 * pp.sig_perp;
  pv.sigbar_w_d = sqrt(sq2 + sw2);
  pv.chi_w_d = chi_w;
  // largest cell-wall range: face on sqrt(sig_par^2 + sig_w^2), side on sigbar_w
  pv.sigw_max = (float)(fmax(sqrt(sq2 + sw2), sqrt(sp2 + sw2)) * 1.0001);
}

extern "C" int bl_particles_set(bl_ctx *c, int n, const bl_particle_params *pp, const double *X, const double *q,
                                const double *V, const double *L) {
  if (!c || n < 0 || !pp) return BL_EINVAL;
  if (c->sticky) return c->sticky;
  if (n > 0 && (!X || !q || !V || !L)) return fail(c, BL_EINVAL, "null state array");
  if (n > 0 && (!(pp->R_par > 0) || !(pp->R_perp > 0) || !(pp->r_cut > 0) || !(pp->rho_p > 0) ||
                !(pp->sig_par > 0) || !(pp->sig_perp > 0) || !(pp->R_par < 1e4) || !(pp->R_perp < 1e4) ||
                !(pp->sig_w >= 0) || !(pp->eps >= 0) || !(pp->eps_w >= 0)))
    return fail(c, BL_EINVAL, "bad cell parameters");
  if (pp->move_particles < 0 || pp->move_particles > 2) return fail(c, BL_EINVAL, "move_particles not in 0..2");
  if (n > 0) {
    // the owner search covers one cell-list bin around a node (bins are at
    // least r_cut wide), and a cell must not reach half a periodic length
    const double rmax = fmax(pp->R_par, pp->R_perp);
    if (!(pp->r_cut >= rmax + 1.0)) return fail(c, BL_EINVAL, "r_cut < max(R_par, R_perp) + 1");
    const int dims[3] = {c->lv.nx, c->lv.ny, c->lv.nz};
    for (int k = 0; k < 3; ++k)
      if (c->lv.per[k] && !((double)dims[k] >= 2.0 * rmax + 4.0))
        return fail(c, BL_EINVAL, "periodic length %d < 2 max(R) + 4", dims[k]);
  }
  const bool first = n != c->np || c->np == 0;
  // a new set of cells clears the old cells and rebuilds the geometry, which
  // drops pending terms: they go to the populations first.  A re-placement
  // keeps them: fluid that stays fluid gets its term in the next sweep (which
  // reads every fluid node's pending velocity), and the resolve counts that
  // of fluid it covers in the impulses
  if (first && flush_pending(c)) return c->sticky;
  // the graphs hold the cell arrays' pointers and the cell constants by
  // value: they stay valid for a re-placement with the same arrays and
  // parameters (their keys, parity and kinematics buffer, are checked)
  if (first || memcmp(&c->pp, pp, sizeof(bl_particle_params)) != 0) drop_graph(c);
  if (first) {
    // cells of a previous call become resting fluid
    launch_clear_cells(c->dtype, c->lv, c->parity, c->stream, &c->launches);
    if (check_launch(c, "clear cells")) return c->sticky;
    CU(cudaStreamSynchronize(c->stream));
    free_particles(c);
    c->pp = *pp;
    if (!c->sweep_fixed) c->lv.sweep = auto_sweep(c);
    if (n == 0) {
      launch_geometry(c->lv, c->pv, c->stream, &c->launches);
      if (check_launch(c, "geometry")) return c->sticky;
      CU(cudaStreamSynchronize(c->stream));
      return BL_OK;
    }
    if (alloc_particles(c, n)) return c->sticky;
    if (!c->sweep_fixed) c->lv.sweep = auto_sweep(c);
    if (c->mlp && alloc_pairbuf(c)) return c->sticky;
  } else {
    c->pp = *pp;
  }
  fill_particle_constants(c);
  std::vector<double> st(13 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    for (int k = 0; k < 3; ++k) {
      st[13 * i + k] = X[3 * i + k];
      st[13 * i + 7 + k] = V[3 * i + k];
      st[13 * i + 10 + k] = L[3 * i + k];
    }
    for (int k = 0; k < 4; ++k) st[13 * i + 3 + k] = q[4 * i + k];
    const int dims[3] = {c->lv.nx, c->lv.ny, c->lv.nz};
    for (int k = 0; k < 3; ++k)
      if (!(X[3 * i + k] >= 0.0 && X[3 * i + k] < (double)dims[k]))
        return fail(c, BL_EINVAL, "cell %d: X outside [0, N)", i);
  }
  CU(cudaMemcpyAsync(c->pv.stage, st.data(), sizeof(double) * st.size(), cudaMemcpyHostToDevice, c->stream));
  launch_set_state(c->lv, c->pv, first ? 1 : 2, c->stream, &c->launches);
  // the search for new owners of nodes that a cell leaves uses the cell list
  // of the new positions
  if (!first) launch_cell_list(c->lv, c->pv, c->cl, c->stream, &c->launches);
  launch_claims(c->lv, c->pv, c->claim, c->chg, first ? 1 : 2, c->stream, &c->launches);
  launch_resolve_fill(c->dtype, c->lv, c->pv, c->cl, c->claim, c->chg, c->parity, first ? 0 : 1, c->stream,
                      &c->launches);
  // neighbour words: the whole lattice after a first placement; after a
  // re-placement only around the nodes resolve changed (every step starts by
  // summing the contact links of the current owner map)
  if (first) launch_geometry(c->lv, c->pv, c->stream, &c->launches);
  else launch_nbm_update(c->lv, c->pv, c->chg, c->stream, &c->launches);
  std::swap(c->pv.kin, c->pv.kin_next);
  if (check_launch(c, "particles_set")) return c->sticky;
  // a first placement waits (device errors surface here); a re-placement
  // returns at once like bl_step: the state was staged by the copy call
  // (pageable host memory), and device errors surface at the next bl_sync
  if (first) CU(cudaStreamSynchronize(c->stream));
  return BL_OK;
}

// one step on stream st (the caller's stream, or the graph stream while a
// graph is captured)
static int enqueue_step(bl_ctx *c, cudaStream_t st) {
  int slot;
  // with timing enabled the sweep runs first and alone, the side streams
  // after it, so that its event time is the kernel's own and not its share
  // of the GPU beside the cell list and the potentials (the step's graph, which
  // is what a timed run replays, keeps them beside each other)
  const bool sweep_alone = c->timing != 0;
  if (sweep_alone) {
    group_begin(c, 0, &slot, st);
    launch_lb_step(c->dtype, c->lv, c->parity, c->wacc, c->status, st);
    group_end(c, slot, st);
    c->launches++;
    if (c->le_on) launch_lees_edwards(c->dtype, c->lv, c->le, c->parity, st, &c->launches);
  }
  if (c->np > 0) {
    // cell list and potentials from the state at t, beside the sweep; on a
    // second side stream the contact sums of the current owner map
    cudaEventRecord(c->ev_fork, st);
    cudaStreamWaitEvent(c->side, c->ev_fork, 0);
    cudaStreamWaitEvent(c->side2, c->ev_fork, 0);
    group_begin(c, 4, &slot, c->side2);
    launch_contacts(c->lv, c->pv, c->side2, &c->launches);
    group_end(c, slot, c->side2);
    cudaEventRecord(c->ev_join3, c->side2);
    group_begin(c, 1, &slot, c->side);
    launch_cell_list(c->lv, c->pv, c->cl, c->side, &c->launches);
    group_end(c, slot, c->side);
    group_begin(c, 2, &slot, c->side);
    launch_forces(c->lv, c->pv, c->cl, c->sbits, c->side, &c->launches);
    if (c->mlp)
      launch_mlp_correction(c->lv, c->pv, c->cl, c->pb, c->gap_lo, c->gap_cut, c->speed_lo, c->speed_hi, c->mlp,
                            c->side, &c->launches);
    group_end(c, slot, c->side);
    cudaEventRecord(c->ev_join, c->side);
  }
  if (!sweep_alone) {
    group_begin(c, 0, &slot, st);
    launch_lb_step(c->dtype, c->lv, c->parity, c->wacc, c->status, st);
    group_end(c, slot, st);
    c->launches++;
    if (c->le_on) launch_lees_edwards(c->dtype, c->lv, c->le, c->parity, st, &c->launches);
  }
  if (c->np > 0) {
    cudaStreamWaitEvent(st, c->ev_join, 0);
    cudaStreamWaitEvent(st, c->ev_join3, 0);
    group_begin(c, 3, &slot, st);
    launch_sums_solve(c->dtype, c->lv, c->pv, c->parity, st, &c->launches);
    group_end(c, slot, st);
    // the claims need only the solve: beside the pending C of the records
    cudaEventRecord(c->ev_fork2, st);
    cudaStreamWaitEvent(c->side, c->ev_fork2, 0);
    group_begin(c, 3, &slot, c->side);
    launch_claims(c->lv, c->pv, c->claim, c->chg, 0, c->side, &c->launches);
    group_end(c, slot, c->side);
    cudaEventRecord(c->ev_join2, c->side);
    group_begin(c, 3, &slot, st);
    launch_link_pending(c->dtype, c->lv, c->pv, c->parity, st, &c->launches);
    group_end(c, slot, st);
    cudaStreamWaitEvent(st, c->ev_join2, 0);
    group_begin(c, 4, &slot, st);
    launch_resolve_fill(c->dtype, c->lv, c->pv, c->cl, c->claim, c->chg, c->parity ^ 1, 1, st, &c->launches);
    launch_nbm_update(c->lv, c->pv, c->chg, st, &c->launches);
    group_end(c, slot, st);
    std::swap(c->pv.kin, c->pv.kin_next);
  }
  c->parity ^= 1;
  return check_launch(c, "step");
}

static void drop_graph(bl_ctx *c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  for (int k = 0; k < 2; ++k) {
    if (c->g1exec[k]) cudaGraphExecDestroy(c->g1exec[k]);
    c->g1exec[k] = nullptr;
  }
  c->epoch++;
}

// the graph of two steps from the current parity and cell state
static int capture_graph(bl_ctx *c) {
  drop_graph(c);
  const int64_t l0 = c->launches;
  const int par = c->parity;
  const void *kin = c->pv.kin;
  cudaGraph_t g = nullptr;
  CU(cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_step(c, c->gstream);
  if (rc == BL_OK) rc = enqueue_step(c, c->gstream);
  cudaError_t e = cudaStreamEndCapture(c->gstream, &g);
  // capturing records the kernels without running them: the two steps
  // flipped the parity and swapped the kinematics buffers twice, but an
  // aborted capture may have stopped after one
  c->parity = par;
  if (c->pv.kin != (const float4 *)kin) std::swap(c->pv.kin, c->pv.kin_next);
  c->g_launches = c->launches - l0;
  c->launches = l0;
  if (rc != BL_OK) return rc;
  if (e != cudaSuccess) return fail(c, BL_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&c->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->gexec = nullptr;
    return fail(c, BL_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  c->g_parity = par;
  c->g_kin = kin;
  return BL_OK;
}

// the graph of one step from the current parity and cell state
static int capture_graph1(bl_ctx *c) {
  const int par = c->parity;
  if (c->g1exec[par]) cudaGraphExecDestroy(c->g1exec[par]);
  c->g1exec[par] = nullptr;
  const int64_t l0 = c->launches;
  const void *kin = c->pv.kin;
  cudaGraph_t g = nullptr;
  CU(cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_step(c, c->gstream);
  cudaError_t e = cudaStreamEndCapture(c->gstream, &g);
  c->parity = par;  // capturing ran nothing: undo the step's host-side flips
  if (c->pv.kin != (const float4 *)kin) std::swap(c->pv.kin, c->pv.kin_next);
  c->g1_launches[par] = c->launches - l0;
  c->launches = l0;
  if (rc != BL_OK) return rc;
  if (e != cudaSuccess) return fail(c, BL_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&c->g1exec[par], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->g1exec[par] = nullptr;
    return fail(c, BL_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  c->g1kin[par] = kin;
  return BL_OK;
}

extern "C" int bl_step(bl_ctx *c, int nsteps) {
  if (!c || nsteps < 0) return BL_EINVAL;
  if (c->sticky) return c->sticky;
  int s = 0;
  if (!c->timing && nsteps >= 2) {
    // pairs of steps as one graph launch
    if (!c->gexec || c->g_parity != c->parity || c->g_kin != (const void *)c->pv.kin)
      if (capture_graph(c)) return c->sticky;
    CU(cudaEventRecord(c->ev_fork, c->stream));
    CU(cudaStreamWaitEvent(c->gstream, c->ev_fork, 0));
    for (; s + 2 <= nsteps; s += 2) {
      CU(cudaGraphLaunch(c->gexec, c->gstream));
      c->launches += c->g_launches;
    }
    CU(cudaEventRecord(c->ev_join, c->gstream));
    CU(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  }
  if (!c->timing && s < nsteps) {
    // a last single step as a one-step graph
    const int par = c->parity;
    if (!c->g1exec[par] || c->g1kin[par] != (const void *)c->pv.kin)
      if (capture_graph1(c)) return c->sticky;
    CU(cudaEventRecord(c->ev_fork, c->stream));
    CU(cudaStreamWaitEvent(c->gstream, c->ev_fork, 0));
    CU(cudaGraphLaunch(c->g1exec[par], c->gstream));
    c->launches += c->g1_launches[par];
    CU(cudaEventRecord(c->ev_join, c->gstream));
    CU(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    c->parity ^= 1;  // what the step does on the host
    if (c->np > 0) std::swap(c->pv.kin, c->pv.kin_next);
    ++s;
  }
  for (; s < nsteps; ++s)
    if (enqueue_step(c, c->stream)) return c->sticky;
  return BL_OK;
}

extern "C" int bl_lees_edwards_set(bl_ctx *c, double U, double d_reflect) {
  if (!c || !(fabs(U) < 0.3) || !(d_reflect == d_reflect)) return BL_EINVAL;
  if (c->sticky) return c->sticky;
  if (!c->lv.per[0] || !c->lv.per[1] || !c->lv.per[2])
    return fail(c, BL_EINVAL, "Lees-Edwards shear needs every axis periodic");
  if (c->masked) return fail(c, BL_ESTATE, "Lees-Edwards shear with a wall mask (its planes must hold fluid)");
  const size_t M = (size_t)c->lv.ny * c->lv.nz;
  if (!c->le_on) {
    if (cudaMalloc(&c->lv.le_mom, sizeof(float4) * 2 * M) != cudaSuccess ||
        cudaMalloc(&c->le.T, sizeof(float) * 10 * M) != cudaSuccess ||
        cudaMalloc(&c->le.D, sizeof(double)) != cudaSuccess || cudaMalloc(&c->le.t, sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&c->le.P, sizeof(double)) != cudaSuccess || cudaMalloc(&c->le.n, sizeof(long long)) != cudaSuccess)
      return fail(c, BL_ENOMEM, "Lees-Edwards buffers");
  }
  CU(cudaMemsetAsync(c->le.t, 0, sizeof(long long), c->stream));
  CU(cudaMemsetAsync(c->le.P, 0, sizeof(double), c->stream));
  CU(cudaMemsetAsync(c->le.n, 0, sizeof(long long), c->stream));
  c->le.U = U;
  c->le_on = 1;
  c->le_dr_req = d_reflect;
  if (c->np > 0) fill_particle_constants(c);
  drop_graph(c);  // the graphs hold the views by value
  return BL_OK;
}

extern "C" int bl_lees_edwards_get(bl_ctx *c, double *P_sum, int64_t *steps) {
  if (!c || !P_sum || !steps) return BL_EINVAL;
  if (c->sticky) return c->sticky;
  if (!c->le_on) return fail(c, BL_ESTATE, "no Lees-Edwards shear set");
  long long n = 0;
  CU(cudaMemcpyAsync(P_sum, c->le.P, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(&n, c->le.n, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  *steps = (int64_t)n;
  return read_status(c);
}

static int read_status(bl_ctx *c) {
  int st = 0;
  CU(cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (st & ST_UNSTABLE) return fail(c, BL_EUNSTABLE, "unstable: rho <= 0, NaN or |u| >= 0.3 at some node, or a cell speed >= 0.5");
  if (st & ST_OVERFLOW) return fail(c, BL_EOVERFLOW, "internal list overflow");
  if (st & ST_BARRIER) return fail(c, BL_EBARRIER, "a bounded wait for asynchronous copies timed out");
  if (st & ST_LEPLANE) return fail(c, BL_ESTATE, "a node beside the Lees-Edwards plane is not fluid (a cell reached it)");
  return BL_OK;
}

extern "C" int bl_sync(bl_ctx *c) {
  if (!c) return BL_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, BL_ECUDA, "stream: %s", cudaGetErrorString(e));
  if (c->sticky) return c->sticky;
  return read_status(c);
}

extern "C" int bl_fields_get(bl_ctx *c, double *rho, double *u, int32_t *owner, int on_device) {
  if (!c) return BL_EINVAL;
  if (c->sticky) return c->sticky;
  if (flush_pending(c)) return c->sticky;
  const size_t N = c->lv.N;
  if (on_device) {
    launch_fields(c->dtype, c->lv, c->parity, rho, u, owner, c->stream);
    c->launches++;
    return check_launch(c, "fields");
  }
  if (ensure_scratch(c, N * sizeof(double) * 4 + N * sizeof(int32_t))) return c->sticky;
  double *drho = c->scratch, *du = c->scratch + N;
  int32_t *down = (int32_t *)(c->scratch + 4 * N);
  launch_fields(c->dtype, c->lv, c->parity, drho, du, down, c->stream);
  c->launches++;
  if (check_launch(c, "fields")) return c->sticky;
  if (rho) CU(cudaMemcpyAsync(rho, drho, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (u) CU(cudaMemcpyAsync(u, du, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (owner) CU(cudaMemcpyAsync(owner, down, N * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return BL_OK;
}

static int copy_n3(bl_ctx *c, double *dst, const double *src, int comps) {
  if (!dst || !src || c->np == 0) return BL_OK;
  CU(cudaMemcpyAsync(dst, src, sizeof(double) * comps * (size_t)c->np, cudaMemcpyDeviceToHost, c->stream));
  return BL_OK;
}

extern "C" int bl_forces_get(bl_ctx *c, double *F, double *T, double *X, double *q, double *V, double *L) {
  if (!c) return BL_EINVAL;
  if (c->sticky) return c->sticky;
  if (copy_n3(c, F, c->pv.Ftot, 3) || copy_n3(c, T, c->pv.Ttot, 3) || copy_n3(c, X, c->pv.X, 3) ||
      copy_n3(c, q, c->pv.q, 4) || copy_n3(c, V, c->pv.V, 3) || copy_n3(c, L, c->pv.L, 3))
    return c->sticky;
  CU(cudaStreamSynchronize(c->stream));
  return BL_OK;
}

extern "C" int bl_force_parts_get(bl_ctx *c, double *Fh, double *Th, double *Fp, double *Tp, double *Om, double *PF,
                                  double *PT) {
  if (!c) return BL_EINVAL;
  if (c->sticky) return c->sticky;
  if (copy_n3(c, Fh, c->pv.Flink, 3) || copy_n3(c, Th, c->pv.Tlink, 3) || copy_n3(c, Fp, c->pv.Fpot, 3) ||
      copy_n3(c, Tp, c->pv.Tpot, 3) || copy_n3(c, Om, c->pv.Om, 3) || copy_n3(c, PF, c->pv.PF, 3) ||
      copy_n3(c, PT, c->pv.PT, 3))
    return c->sticky;
  CU(cudaStreamSynchronize(c->stream));
  return BL_OK;
}

extern "C" int bl_wall_momentum_get(bl_ctx *c, double *wallmom) {
  if (!c || !wallmom) return BL_EINVAL;
  if (c->sticky) return c->sticky;
  double F[bl::NWALL * 3];
  long long K[bl::NWALL * 3];
  CU(cudaMemcpyAsync(F, c->wacc.F, sizeof(F), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(K, c->wacc.K, sizeof(K), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  CU(cudaMemsetAsync(c->wacc.F, 0, sizeof(F), c->stream));
  CU(cudaMemsetAsync(c->wacc.K, 0, sizeof(K), c->stream));
  for (int i = 0; i < bl::NWALL * 3; ++i) wallmom[i] = F[i] + c->lp.rho0 / 18.0 * (double)K[i];
  return BL_OK;
}

extern "C" int bl_populations_get(bl_ctx *c, double *pop) {
  if (!c || !pop) return BL_EINVAL;
  if (c->sticky) return c->sticky;
  if (flush_pending(c)) return c->sticky;
  const size_t bytes = sizeof(double) * bl::Q * (size_t)c->lv.N;
  if (ensure_scratch(c, bytes)) return c->sticky;
  launch_pop_io(c->dtype, c->lv, c->parity, c->scratch, 0, c->stream);
  c->launches++;
  if (check_launch(c, "populations get")) return c->sticky;
  CU(cudaMemcpyAsync(pop, c->scratch, bytes, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return BL_OK;
}

extern "C" int bl_populations_set(bl_ctx *c, const double *pop) {
  if (!c || !pop) return BL_EINVAL;
  if (c->sticky) return c->sticky;
  if (flush_pending(c)) return c->sticky;  // (the set overwrites them: nothing may pend after it)
  const size_t bytes = sizeof(double) * bl::Q * (size_t)c->lv.N;
  if (ensure_scratch(c, bytes)) return c->sticky;
  CU(cudaMemcpyAsync(c->scratch, pop, bytes, cudaMemcpyHostToDevice, c->stream));
  launch_pop_io(c->dtype, c->lv, c->parity, c->scratch, 1, c->stream);
  c->launches++;
  if (check_launch(c, "populations set")) return c->sticky;
  CU(cudaStreamSynchronize(c->stream));
  return BL_OK;
}

static int links_get(bl_ctx *c, int contact, int32_t *out, int64_t cap, int64_t *count) {
  if (!c || !count || cap < 0) return BL_EINVAL;
  if (c->sticky) return c->sticky;
  const unsigned nb = links_blocks(c->lv);
  int *bc = nullptr, *off = nullptr;
  int32_t *dout = nullptr;
  CU(cudaMalloc(&bc, sizeof(int) * nb));
  CU(cudaMalloc(&off, sizeof(int) * nb));
  launch_links(c->lv, contact, 0, bc, nullptr, nullptr, 0, c->stream);
  c->launches++;
  std::vector<int> cnt(nb), o(nb);
  CU(cudaMemcpyAsync(cnt.data(), bc, sizeof(int) * nb, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  long long tot = 0;
  for (unsigned b = 0; b < nb; ++b) {
    o[b] = (int)tot;
    tot += cnt[b];
  }
  *count = tot;
  if (tot > 0 && out && cap > 0) {
    CU(cudaMemcpyAsync(off, o.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMalloc(&dout, sizeof(int32_t) * 3 * (size_t)tot));
    launch_links(c->lv, contact, 1, nullptr, off, dout, tot, c->stream);
    c->launches++;
    const long long ncopy = tot < cap ? tot : cap;
    CU(cudaMemcpyAsync(out, dout, sizeof(int32_t) * 3 * (size_t)ncopy, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
  }
  cudaFree(bc);
  cudaFree(off);
  if (dout) cudaFree(dout);
  return check_launch(c, "links");
}

extern "C" int bl_boundary_links_get(bl_ctx *c, int32_t *out, int64_t cap, int64_t *count) {
  return links_get(c, 0, out, cap, count);
}

extern "C" int bl_contact_links_get(bl_ctx *c, int32_t *out, int64_t cap, int64_t *count) {
  return links_get(c, 1, out, cap, count);
}

extern "C" int bl_cell_links_get(bl_ctx *c, int32_t *out, int64_t cap, int64_t *count) {
  if (!c || !count || cap < 0) return BL_EINVAL;
  if (c->sticky) return c->sticky;
  *count = 0;
  if (c->np == 0) return BL_OK;
  // the link records of the last sweep, as the step's link sums read them
  const int n = c->np, capr = c->lv.rec_cap;
  std::vector<int> cnt(n);
  std::vector<float4> rec((size_t)n * capr * 2);
  CU(cudaMemcpyAsync(cnt.data(), c->pv.rec_last, sizeof(int) * n, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(rec.data(), c->lv.rec, sizeof(float4) * rec.size(), cudaMemcpyDeviceToHost, c->stream));
  if (read_status(c)) return c->sticky;
  struct Link {
    long long node;
    int r, p;
  };
  std::vector<Link> links;
  for (int p = 0; p < n; ++p) {
    for (int i = 0; i < cnt[p] && i < capr; ++i) {
      const float4 r0 = rec[2 * ((size_t)p * capr + i)];
      uint32_t node, mask;
      memcpy(&node, &r0.x, 4);
      memcpy(&mask, &r0.y, 4);
      for (int r = 1; r < bl::Q; ++r)
        if (mask & (1u << r)) links.push_back(Link{(long long)node, r, p});
    }
  }
  std::sort(links.begin(), links.end(), [](const Link &a, const Link &b) {
    return a.node != b.node ? a.node < b.node : (a.r != b.r ? a.r < b.r : a.p < b.p);
  });
  *count = (int64_t)links.size();
  if (out)
    for (int64_t k = 0; k < (int64_t)links.size() && k < cap; ++k) {
      out[3 * k] = (int32_t)links[k].node;
      out[3 * k + 1] = links[k].r;
      out[3 * k + 2] = links[k].p;
    }
  return BL_OK;
}

extern "C" int bl_cell_list_get(bl_ctx *c, int32_t nb[3], int32_t *start, int32_t *ids) {
  if (!c || !nb) return BL_EINVAL;
  if (c->sticky) return c->sticky;
  if (c->np == 0) return fail(c, BL_ESTATE, "no cells");
  for (int k = 0; k < 3; ++k) nb[k] = c->cl.nb[k];
  if (!start && !ids) return BL_OK;
  launch_cell_list(c->lv, c->pv, c->cl, c->stream, &c->launches);
  if (check_launch(c, "cell list")) return c->sticky;
  if (start)
    CU(cudaMemcpyAsync(start, c->cl.start, sizeof(int32_t) * (c->cl.nbins + 1), cudaMemcpyDeviceToHost, c->stream));
  if (ids) CU(cudaMemcpyAsync(ids, c->cl.ids, sizeof(int32_t) * c->np, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return BL_OK;
}

extern "C" int bl_timing_enable(bl_ctx *c, int enable) {
  if (!c) return BL_EINVAL;
  c->timing = enable ? 1 : 0;
  return BL_OK;
}

extern "C" int bl_timing_read(bl_ctx *c, double *ms, int64_t *count, int ngroups) {
  if (!c || ngroups < 0) return BL_EINVAL;
  if (harvest_timing(c)) return c->sticky;
  for (int g = 0; g < ngroups && g < NGROUPS; ++g) {
    if (ms) ms[g] = c->t_ms[g];
    if (count) count[g] = c->t_cnt[g];
  }
  for (int g = 0; g < NGROUPS; ++g) {
    c->t_ms[g] = 0.0;
    c->t_cnt[g] = 0;
  }
  return BL_OK;
}

extern "C" int64_t bl_launch_count(const bl_ctx *c) { return c ? c->launches : 0; }

extern "C" const char *bl_last_error(const bl_ctx *c) { return c ? c->err : "null context"; }

// ---------------------------------------------------------------------------
// learned near-contact correction

extern "C" int bl_mlp_attach_range(bl_ctx *c, bl_mlp *m, double gap_lo, double gap_hi, double speed_lo,
                                   double speed_hi) {
  if (!c) return BL_EINVAL;
  if (c->sticky) return c->sticky;
  if (m && !(gap_lo < gap_hi && gap_hi > -1e3 && gap_hi < 1e3 && gap_lo < 1e3 && speed_lo <= speed_hi &&
             speed_lo >= 0.0))
    return fail(c, BL_EINVAL, "gap or speed range");
  drop_graph(c);
  c->mlp = m;
  c->gap_lo = gap_lo < -1e30 ? -3.0e38f : (float)gap_lo;
  c->gap_cut = (float)gap_hi;
  c->speed_lo = (float)speed_lo;
  c->speed_hi = speed_hi > 1e30 ? 3.0e38f : (float)speed_hi;
  if (m && alloc_pairbuf(c)) return c->sticky;
  return BL_OK;
}

extern "C" int bl_mlp_attach(bl_ctx *c, bl_mlp *m, double gap_cut) {
  return bl_mlp_attach_range(c, m, -1e300, gap_cut, 0.0, 1e300);
}

extern "C" int bl_pair_features(bl_ctx *c, const int32_t *pairs, int n, float *out) {
  if (!c || n < 0 || (n > 0 && (!pairs || !out))) return BL_EINVAL;
  if (c->sticky) return c->sticky;
  launch_pair_features(c->lv, c->pv, reinterpret_cast<const int2 *>(pairs), n, out, c->stream);
  c->launches += n > 0;
  return check_launch(c, "pair features");
}

// ---------------------------------------------------------------------------
// autotuning of the sweep variant

extern "C" int bl_autotune(bl_ctx *c, int trial_steps, int *choice) {
  if (!c || trial_steps < 2) return BL_EINVAL;
  if (c->sticky) return c->sticky;
  if (c->timing) return fail(c, BL_ESTATE, "bl_autotune with timing enabled");
  // candidate variants the storage type and the row length allow
  int cand[6], nvar = 0;
  cand[nvar++] = 0;
  if (c->dtype == BL_STORE_F32) {
    cand[nvar++] = 1;
    cand[nvar++] = 2;
  }
  if (c->lv.nx % (c->dtype == BL_STORE_F32 ? 4 : 8) == 0) {
    cand[nvar++] = 3;
    cand[nvar++] = 4;
    cand[nvar++] = 5;
  }
  int best = 0;
  float best_ms = 0.f;
  cudaEvent_t a, b;
  CU(cudaEventCreate(&a));
  CU(cudaEventCreate(&b));
  int rc = BL_OK;
  for (int iv = 0; iv < nvar && rc == BL_OK; ++iv) {
    const int v = cand[iv];
    drop_graph(c);  // the graph holds the lattice view, variant included
    c->lv.sweep = v;
    if ((rc = bl_step(c, 2)) != BL_OK) break;  // capture + warm-up
    cudaEventRecord(a, c->stream);
    if ((rc = bl_step(c, trial_steps & ~1)) != BL_OK) break;
    cudaEventRecord(b, c->stream);
    if (cudaEventSynchronize(b) != cudaSuccess) {
      rc = fail(c, BL_ECUDA, "autotune timing");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (iv == 0 || ms < best_ms) {
      best = v;
      best_ms = ms;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  drop_graph(c);
  c->lv.sweep = best;
  c->sweep_fixed = 1;
  if (choice) *choice = best;
  if (rc != BL_OK) return rc;
  return read_status(c);
}

extern "C" int bl_sweep_variant(bl_ctx *c, int variant) {
  if (!c || variant < 0 || variant > 5) return BL_EINVAL;
  if (c->sticky) return c->sticky;
  if ((variant == 1 || variant == 2) && c->dtype != BL_STORE_F32) return BL_EINVAL;
  drop_graph(c);
  c->lv.sweep = variant;
  c->sweep_fixed = 1;
  return BL_OK;
}

// ---------------------------------------------------------------------------
// ensembles: independent contexts advanced together by one graph whose
// branches are the members' steps

struct bl_ens {
  std::vector<bl_ctx *> m;
  cudaStream_t stream;  // the caller's stream of the ensemble
  cudaStream_t cap;     // internal stream the graph is captured and replayed on
  cudaEvent_t ev_fork, ev_join;
  std::vector<cudaEvent_t> ev_m;
  cudaGraphExec_t gexec;
  std::vector<int> g_parity, g_epoch;
  std::vector<const void *> g_kin;
  std::vector<int64_t> g_launches;
  int sticky;
};

static void ens_drop(bl_ens *e) {
  if (e->gexec) cudaGraphExecDestroy(e->gexec);
  e->gexec = nullptr;
}

static bool ens_valid(const bl_ens *e) {
  if (!e->gexec) return false;
  for (size_t i = 0; i < e->m.size(); ++i) {
    const bl_ctx *c = e->m[i];
    if (c->parity != e->g_parity[i] || (const void *)c->pv.kin != e->g_kin[i] || c->epoch != e->g_epoch[i])
      return false;
  }
  return true;
}

static int ens_capture(bl_ens *e) {
  ens_drop(e);
  const size_t n = e->m.size();
  std::vector<int64_t> l0(n);
  for (size_t i = 0; i < n; ++i) {
    bl_ctx *c = e->m[i];
    e->g_parity[i] = c->parity;
    e->g_kin[i] = c->pv.kin;
    e->g_epoch[i] = c->epoch;
    l0[i] = c->launches;
  }
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return BL_ECUDA;
  int rc = BL_OK;
  cudaEventRecord(e->ev_fork, e->cap);
  for (size_t i = 0; i < n && rc == BL_OK; ++i) {
    bl_ctx *c = e->m[i];
    cudaStreamWaitEvent(c->gstream, e->ev_fork, 0);
    rc = enqueue_step(c, c->gstream);
    if (rc == BL_OK) rc = enqueue_step(c, c->gstream);
    cudaEventRecord(e->ev_m[i], c->gstream);
    cudaStreamWaitEvent(e->cap, e->ev_m[i], 0);
  }
  const cudaError_t err = cudaStreamEndCapture(e->cap, &g);
  for (size_t i = 0; i < n; ++i) {  // capturing ran nothing: restore the members' step state
    bl_ctx *c = e->m[i];
    c->parity = e->g_parity[i];
    if ((const void *)c->pv.kin != e->g_kin[i]) std::swap(c->pv.kin, c->pv.kin_next);
    e->g_launches[i] = c->launches - l0[i];
    c->launches = l0[i];
  }
  if (rc != BL_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (err != cudaSuccess) return BL_ECUDA;
  const cudaError_t ie = cudaGraphInstantiate(&e->gexec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    e->gexec = nullptr;
    return BL_ECUDA;
  }
  return BL_OK;
}

extern "C" int bl_ensemble_create(bl_ens **out, bl_ctx *const *ctxs, int n, void *cuda_stream) {
  if (!out) return BL_EINVAL;
  *out = nullptr;
  if (!ctxs || n < 1) return BL_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return BL_EINVAL;
    if (ctxs[i]->sticky) return ctxs[i]->sticky;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return BL_EINVAL;
  }
  bl_ens *e = new bl_ens();
  e->m.assign(ctxs, ctxs + n);
  e->stream = (cudaStream_t)cuda_stream;
  e->g_parity.assign(n, 0);
  e->g_epoch.assign(n, 0);
  e->g_kin.assign(n, nullptr);
  e->g_launches.assign(n, 0);
  e->ev_m.assign(n, nullptr);
  bool ok = cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&e->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&e->ev_join, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < n && ok; ++i) ok = cudaEventCreateWithFlags(&e->ev_m[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    bl_ensemble_destroy(e);
    return BL_ECUDA;
  }
  *out = e;
  return BL_OK;
}

extern "C" int bl_ensemble_step(bl_ens *e, int nsteps) {
  if (!e || nsteps < 0) return BL_EINVAL;
  if (e->sticky) return e->sticky;
  for (bl_ctx *c : e->m) {
    if (c->sticky) return e->sticky = c->sticky;
    if (c->timing) return e->sticky = BL_ESTATE;
  }
  int s = 0;
  if (nsteps >= 2) {
    if (!ens_valid(e)) {
      const int rc = ens_capture(e);
      if (rc != BL_OK) return e->sticky = rc;
    }
    // every member's prior work, then the graph, then every member's stream
    for (size_t i = 0; i < e->m.size(); ++i) {
      cudaEventRecord(e->ev_m[i], e->m[i]->stream);
      cudaStreamWaitEvent(e->cap, e->ev_m[i], 0);
    }
    cudaEventRecord(e->ev_fork, e->stream);
    cudaStreamWaitEvent(e->cap, e->ev_fork, 0);
    for (; s + 2 <= nsteps; s += 2) {
      if (cudaGraphLaunch(e->gexec, e->cap) != cudaSuccess) return e->sticky = BL_ECUDA;
      for (size_t i = 0; i < e->m.size(); ++i) e->m[i]->launches += e->g_launches[i];
    }
    cudaEventRecord(e->ev_join, e->cap);
    cudaStreamWaitEvent(e->stream, e->ev_join, 0);
    for (bl_ctx *c : e->m) cudaStreamWaitEvent(c->stream, e->ev_join, 0);
  }
  for (; s < nsteps; ++s)
    for (bl_ctx *c : e->m) {
      const int rc = bl_step(c, 1);
      if (rc != BL_OK) return e->sticky = rc;
    }
  return BL_OK;
}

extern "C" int bl_ensemble_sync(bl_ens *e) {
  if (!e) return BL_EINVAL;
  int rc = e->sticky;
  for (bl_ctx *c : e->m) {
    const int r = bl_sync(c);
    if (rc == BL_OK) rc = r;
  }
  return rc;
}

extern "C" void bl_ensemble_destroy(bl_ens *e) {
  if (!e) return;
  if (e->cap) cudaStreamSynchronize(e->cap);
  ens_drop(e);
  if (e->cap) cudaStreamDestroy(e->cap);
  if (e->ev_fork) cudaEventDestroy(e->ev_fork);
  if (e->ev_join) cudaEventDestroy(e->ev_join);
  for (cudaEvent_t ev : e->ev_m)
    if (ev) cudaEventDestroy(ev);
  delete e;
}

extern "C" void bl_destroy(bl_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  drop_graph(c);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->gstream) cudaStreamDestroy(c->gstream);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  for (cudaEvent_t e : {c->ev_fork2, c->ev_join2, c->ev_join3})
    if (e) cudaEventDestroy(e);
  if (c->side2) cudaStreamDestroy(c->side2);
  free_particles(c);
  void *ptrs[] = {c->lv.pop, c->lv.owner, c->lv.nbm, c->lv.nbc, c->lv.pu, c->claim, c->status,
                  c->wacc.F, c->wacc.K, c->sbits.bits, c->sbits.rows, c->scratch,
                  c->lv.le_mom, c->le.T, c->le.D, c->le.t, c->le.P, c->le.n};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  delete c;
}
