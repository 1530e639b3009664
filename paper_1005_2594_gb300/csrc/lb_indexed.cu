// lb_indexed.cu -- the indexed lattice of vessel networks: only the fluid
// nodes of a sparse geometry are stored and swept.
//
// The paper closes by pointing out that the method, joined to an indexed LB
// scheme, can take flow through digitised vessel networks, whose lumen fills
// a few per cent of its bounding box.  Here the fluid nodes of a lattice with
// walls (face walls and a wall mask, as for the dense lattice) get compact
// indices in dense node order (x fastest, so that runs along x stay
// contiguous and a warp's reads coalesce), and a table gives each fluid
// node's 18 neighbours: a fluid index, or -1 - w for a wall of id w.  Memory
// and traffic scale with the lumen, not the box.
//
// The sweep is the dense lattice's plasma update (Sec. II: moments, Guo
// forcing, BGK toward the third-order equilibrium, mid-link bounce-back with
// the moving-wall term C of Eq. c, the walls' momentum) on one single AA
// buffer of 19 x Nf slots.  The AA pairing cannot use a wall node's slot for
// a bounce (walls have none), so bounced populations stay in their node's
// own slots:
//   even step: read slot r of i; write f*_r to slot rbar of i (open or wall)
//   odd step:  read direction r from slot rbar of i - c_r, or where i - c_r
//              is a wall from slot r of i; write f*_r to slot r of i + c_r,
//              or where i + c_r is a wall to slot rbar of i
// so that every slot is read and written by one thread per step.  Cells are
// not coupled to the indexed lattice (their owner map, claims and fill work
// on the dense node grid).
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/bloodlb.h"
#include "lb_sweep.cuh"

namespace bl {
namespace {

inline unsigned nblk(unsigned n, unsigned b) { return (n + b - 1) / b; }

struct SparseView {
  unsigned Nf;          // fluid nodes
  void *pop;            // 19 x Nf storage elements, slot r of node i at r Nf + i
  const int32_t *nbr;   // 18 x Nf: neighbour i + c_r at (r - 1) Nf + i, fluid index or -1 - wall id
  const int32_t *dense; // Nf: dense node index of each fluid node
  float wall_vel[NWALL][3];
  float omega, rho0, g[3];
  int *status;
};

#ifndef BL_SPARSE_MINB
#define BL_SPARSE_MINB 3
#endif

template <class S, int PAR, bool FORCE, bool TAU1>
__global__ void __launch_bounds__(256, BL_SPARSE_MINB) k_sparse_step(SparseView sv, WallAcc wa) {
  using D = D3Q19;
  const unsigned Nf = sv.Nf;
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  S *pop = reinterpret_cast<S *>(sv.pop);
  int wkey = -1;
  float wF[3] = {0.f, 0.f, 0.f};
  int wK[3] = {0, 0, 0};
  if (i < Nf) {
    // the neighbour table is read twice, here and for the writes (the second
    // time from L1), so that its 18 entries do not stay live through the
    // collision
    float f[Q];
    f[0] = Store<S>::ld(pop + i);
    sfor<1, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      if constexpr (PAR == 0) {
        f[r] = Store<S>::ld(pop + (size_t)r * Nf + i);
      } else {
        const int s = sv.nbr[(size_t)(D::opp(r) - 1) * Nf + i];  // the node i - c_r
        f[r] = Store<S>::ld(pop + (s >= 0 ? (size_t)D::opp(r) * Nf + (unsigned)s : (size_t)r * Nf + i));
      }
    });
    // moments of the shifted populations: rho = rho_bar + sum f~, j = sum f~ c
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
    sfor<0, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      drho += f[r];
      if constexpr (D::cx(r) != 0) jx += D::cx(r) * f[r];
      if constexpr (D::cy(r) != 0) jy += D::cy(r) * f[r];
      if constexpr (D::cz(r) != 0) jz += D::cz(r) * f[r];
    });
    const float rho = sv.rho0 + drho;
    const float inv = 1.0f / rho;
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    if constexpr (FORCE) {
      Fx = rho * sv.g[0];
      Fy = rho * sv.g[1];
      Fz = rho * sv.g[2];
    }
    const float ux = (jx + 0.5f * Fx) * inv, uy = (jy + 0.5f * Fy) * inv, uz = (jz + 0.5f * Fz) * inv;
    const float uu = ux * ux + uy * uy + uz * uz;
    if (!(rho > 0.f) || !(uu < 0.09f)) atomicOr(sv.status, ST_UNSTABLE);
    const float om = sv.omega, src_w = 1.0f - 0.5f * om, uF = ux * Fx + uy * Fy + uz * Fz;
    // BGK toward w (drho + rho t_r(u)) with the Guo source; at tau = 1 the
    // equilibrium itself
    auto relax = [&](float fr, float w, float t, float cu, float cF) {
      const float feq = w * (drho + fmaf(drho, t, sv.rho0 * t));
      float fs = TAU1 ? feq : fr - om * (fr - feq);
      if constexpr (FORCE) fs += src_w * w * (3.0f * (cF - uF) + 9.0f * cu * cF);
      return fs;
    };
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
    Store<S>::st(pop + i, f[0]);
    sfor<1, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      constexpr int rb = D::opp(r);
      const int t = sv.nbr[(size_t)(r - 1) * Nf + i];
      float v = f[r];
      if (t < 0) {
        // a link into wall w: the population returns along rbar with the
        // moving-wall term C (Eq. c), the wall receives (2 f*_r + C) c_r
        const int w = -1 - t;
        const float C = -(D::m(r) / 6.0f) * rho *
                        (D::cx(r) * sv.wall_vel[w][0] + D::cy(r) * sv.wall_vel[w][1] + D::cz(r) * sv.wall_vel[w][2]);
        const float dp = 2.0f * f[r] + C;
        if (wkey != w && wkey >= 0) {
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
        v += C;
      }
      const size_t dst = (t >= 0 && PAR == 1) ? (size_t)r * Nf + (unsigned)t : (size_t)rb * Nf + i;
      Store<S>::st(pop + dst, v);
    });
  }
  flush_wall_momentum(wa, wkey, wF, wK);
}

// slot from which fluid node i reads direction r in a step of parity par
__device__ __forceinline__ size_t sparse_src(const SparseView &sv, int par, unsigned i, int r) {
  if (par == 0 || r == 0) return (size_t)r * sv.Nf + i;
  const int s = sv.nbr[(size_t)(D3Q19::opp(r) - 1) * sv.Nf + i];
  return s >= 0 ? (size_t)D3Q19::opp(r) * sv.Nf + (unsigned)s : (size_t)r * sv.Nf + i;
}

// moments on the dense grid (zero at walls): rho and u = (j + rho g / 2) / rho
template <class S>
__global__ void k_sparse_fields(SparseView sv, int par, double *rho, double *u) {
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sv.Nf) return;
  const S *pop = reinterpret_cast<const S *>(sv.pop);
  double d = 0.0, j[3] = {0.0, 0.0, 0.0};
  for (int r = 0; r < Q; ++r) {
    const double v = (double)Store<S>::ld(pop + sparse_src(sv, par, i, r));
    d += v;
    j[0] += D3Q19::cx(r) * v;
    j[1] += D3Q19::cy(r) * v;
    j[2] += D3Q19::cz(r) * v;
  }
  const double rh = (double)sv.rho0 + d;
  const unsigned n = (unsigned)sv.dense[i];
  if (rho) rho[n] = rh;
  if (u)
    for (int k = 0; k < 3; ++k) u[3 * (size_t)n + k] = (j[k] + 0.5 * rh * (double)sv.g[k]) / rh;
}

// populations n_r (unshifted) on the dense grid, N x 19, to (0) or from (1) storage
template <class S>
__global__ void k_sparse_pop_io(SparseView sv, int par, double *buf, int to_storage) {
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sv.Nf) return;
  S *pop = reinterpret_cast<S *>(sv.pop);
  const size_t n = (size_t)sv.dense[i];
  for (int r = 0; r < Q; ++r) {
    const double shift = (double)sv.rho0 * D3Q19::m(r) / 36.0;
    const size_t s = sparse_src(sv, par, i, r);
    if (to_storage) Store<S>::st(pop + s, (float)(buf[n * Q + r] - shift));
    else buf[n * Q + r] = (double)Store<S>::ld(pop + s) + shift;
  }
}

template <class S>
__global__ void k_sparse_rest(SparseView sv) {
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sv.Nf) return;
  S *pop = reinterpret_cast<S *>(sv.pop);
  for (int r = 0; r < Q; ++r) Store<S>::st(pop + (size_t)r * sv.Nf + i, 0.0f);
}

template <class S>
void launch_sparse_typed(const SparseView &sv, int par, bool force, bool tau1, const WallAcc &wa, cudaStream_t st) {
  const unsigned b = 256, g = nblk(sv.Nf, b);
#define BL_SP(P_, F_, T_) k_sparse_step<S, P_, F_, T_><<<g, b, 0, st>>>(sv, wa)
  if (par == 0) {
    if (force) { if (tau1) BL_SP(0, true, true); else BL_SP(0, true, false); }
    else { if (tau1) BL_SP(0, false, true); else BL_SP(0, false, false); }
  } else {
    if (force) { if (tau1) BL_SP(1, true, true); else BL_SP(1, true, false); }
    else { if (tau1) BL_SP(1, false, true); else BL_SP(1, false, false); }
  }
#undef BL_SP
}

}  // namespace
}  // namespace bl

using namespace bl;

struct bl_sparse {
  bl_lb_params lp;
  cudaStream_t stream, gstream;
  cudaEvent_t ev_fork, ev_join;
  cudaGraphExec_t gexec;
  int g_parity;
  SparseView sv;
  WallAcc wa;
  int parity;
  int64_t n_dense;
  int sticky;
  char err[256];
  int64_t launches;
  double *scratch;
  size_t scratch_bytes;
};

static int sp_fail(bl_sparse *s, int code, const char *fmt, ...) {
  if (s && s->sticky == BL_OK) {
    s->sticky = code;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(s->err, sizeof(s->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define SPCU(call)                                                                  \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) return sp_fail(s, BL_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// wall id of node (x, y, z): the first walled axis (x, y, z order) whose
// layer holds it, a nonzero mask value k overriding with id k - 1; -1 fluid
static int node_wall(const bl_lb_params *p, const uint8_t *mask, int x, int y, int z) {
  const long long n = (long long)x + (long long)p->nx * ((long long)y + (long long)p->ny * z);
  if (mask && mask[n]) return (int)mask[n] - 1;
  const int c[3] = {x, y, z}, d[3] = {p->nx, p->ny, p->nz};
  for (int k = 0; k < 3; ++k) {
    if (p->periodic[k]) continue;
    if (c[k] == 0) return 2 * k;
    if (c[k] == d[k] - 1) return 2 * k + 1;
  }
  return -1;
}

extern "C" int bl_sparse_index_build(const bl_lb_params *p, const uint8_t *mask, int64_t *n_fluid, int32_t *dense_of,
                                     int32_t *nbr) {
  if (!p || !n_fluid || p->nx < 1 || p->ny < 1 || p->nz < 1) return BL_EINVAL;
  const long long N = (long long)p->nx * p->ny * p->nz;
  if (N >= (1ll << 31)) return BL_EINVAL;
  for (int k = 0; k < 3; ++k) {
    const int n = k == 0 ? p->nx : (k == 1 ? p->ny : p->nz);
    if (!p->periodic[k] && n < 3) return BL_EINVAL;
  }
  if (mask)
    for (long long n = 0; n < N; ++n)
      if (mask[n] > NWALL) return BL_EINVAL;
  std::vector<int32_t> id((size_t)N, -1);
  long long nf = 0;
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        const long long n = (long long)x + (long long)p->nx * ((long long)y + (long long)p->ny * z);
        const int w = node_wall(p, mask, x, y, z);
        id[(size_t)n] = w >= 0 ? -1 - w : (int32_t)nf++;
      }
  const long long prev = *n_fluid;
  *n_fluid = nf;
  if (!dense_of && !nbr) return BL_OK;
  if (prev < nf) return BL_EINVAL;  // the arrays hold fewer nodes than the lattice has
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        const long long n = (long long)x + (long long)p->nx * ((long long)y + (long long)p->ny * z);
        const int32_t i = id[(size_t)n];
        if (i < 0) continue;
        if (dense_of) dense_of[i] = (int32_t)n;
        if (!nbr) continue;
        for (int r = 1; r < Q; ++r) {
          // a fluid node's neighbours lie in the box: a walled axis has wall
          // layers at its ends, a periodic one wraps
          const int xx = (x + D3Q19::cx(r) + p->nx) % p->nx, yy = (y + D3Q19::cy(r) + p->ny) % p->ny,
                    zz = (z + D3Q19::cz(r) + p->nz) % p->nz;
          const long long m = (long long)xx + (long long)p->nx * ((long long)yy + (long long)p->ny * zz);
          nbr[(size_t)(r - 1) * nf + i] = id[(size_t)m];
        }
      }
  return BL_OK;
}

extern "C" void bl_sparse_destroy(bl_sparse *s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  if (s->gstream) cudaStreamDestroy(s->gstream);
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_join) cudaEventDestroy(s->ev_join);
  void *ptrs[] = {s->sv.pop, (void *)s->sv.nbr, (void *)s->sv.dense, s->sv.status, s->wa.F, s->wa.K, s->scratch};
  for (void *q : ptrs)
    if (q) cudaFree(q);
  delete s;
}

static size_t sp_elem(int dtype) { return dtype == BL_STORE_F32 ? 4 : 2; }

static int sp_check(bl_sparse *s, const char *what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return sp_fail(s, BL_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  return BL_OK;
}

static void sp_launch_step(bl_sparse *s, cudaStream_t st, int par) {
  const bool force = s->lp.g[0] != 0.0 || s->lp.g[1] != 0.0 || s->lp.g[2] != 0.0;
  const bool tau1 = s->sv.omega == 1.0f;
  if (s->lp.store_dtype == BL_STORE_F32) launch_sparse_typed<float>(s->sv, par, force, tau1, s->wa, st);
  else if (s->lp.store_dtype == BL_STORE_BF16) launch_sparse_typed<__nv_bfloat16>(s->sv, par, force, tau1, s->wa, st);
  else launch_sparse_typed<__half>(s->sv, par, force, tau1, s->wa, st);
}

extern "C" int bl_sparse_init(bl_sparse **out, const bl_lb_params *p, const uint8_t *mask, void *cuda_stream) {
  if (!out) return BL_EINVAL;
  *out = nullptr;
  if (!p || !(p->tau > 0.5) || !(p->rho0 > 0) || p->store_dtype < 0 || p->store_dtype > 2) return BL_EINVAL;
  int64_t nf = 0;
  int rc = bl_sparse_index_build(p, mask, &nf, nullptr, nullptr);
  if (rc != BL_OK) return rc;
  if (nf < 1 || (unsigned long long)nf * Q >= (1ull << 32)) return BL_EINVAL;
  std::vector<int32_t> dense((size_t)nf), nbr((size_t)nf * 18);
  rc = bl_sparse_index_build(p, mask, &nf, dense.data(), nbr.data());
  if (rc != BL_OK) return rc;
  bl_sparse *s = new bl_sparse();
  s->lp = *p;
  s->stream = (cudaStream_t)cuda_stream;
  s->sticky = BL_OK;
  s->n_dense = (int64_t)p->nx * p->ny * p->nz;
  SparseView &sv = s->sv;
  sv.Nf = (unsigned)nf;
  for (int w = 0; w < NWALL; ++w)
    for (int k = 0; k < 3; ++k) sv.wall_vel[w][k] = (float)p->wall_vel[w][k];
  sv.omega = (float)(1.0 / p->tau);
  sv.rho0 = (float)p->rho0;
  for (int k = 0; k < 3; ++k) sv.g[k] = (float)p->g[k];
  do {
    void *pop = nullptr, *nb = nullptr, *dn = nullptr;
    if (cudaMalloc(&pop, sp_elem(p->store_dtype) * Q * (size_t)nf) != cudaSuccess ||
        cudaMalloc(&nb, sizeof(int32_t) * 18 * (size_t)nf) != cudaSuccess ||
        cudaMalloc(&dn, sizeof(int32_t) * (size_t)nf) != cudaSuccess || cudaMalloc(&sv.status, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&s->wa.F, sizeof(double) * NWALL * 3) != cudaSuccess ||
        cudaMalloc(&s->wa.K, sizeof(long long) * NWALL * 3) != cudaSuccess) {
      sv.pop = pop;
      sv.nbr = (const int32_t *)nb;
      sv.dense = (const int32_t *)dn;
      rc = sp_fail(s, BL_ENOMEM, "indexed lattice");
      break;
    }
    sv.pop = pop;
    sv.nbr = (const int32_t *)nb;
    sv.dense = (const int32_t *)dn;
    if (cudaStreamCreateWithFlags(&s->gstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) != cudaSuccess) {
      rc = sp_fail(s, BL_ECUDA, "streams");
      break;
    }
    if (cudaMemcpyAsync(nb, nbr.data(), sizeof(int32_t) * nbr.size(), cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
        cudaMemcpyAsync(dn, dense.data(), sizeof(int32_t) * dense.size(), cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
        cudaMemsetAsync(sv.status, 0, sizeof(int), s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->wa.F, 0, sizeof(double) * NWALL * 3, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->wa.K, 0, sizeof(long long) * NWALL * 3, s->stream) != cudaSuccess) {
      rc = sp_fail(s, BL_ECUDA, "upload");
      break;
    }
    const unsigned b = 256, g = nblk(sv.Nf, b);
    if (p->store_dtype == BL_STORE_F32) k_sparse_rest<float><<<g, b, 0, s->stream>>>(sv);
    else if (p->store_dtype == BL_STORE_BF16) k_sparse_rest<__nv_bfloat16><<<g, b, 0, s->stream>>>(sv);
    else k_sparse_rest<__half><<<g, b, 0, s->stream>>>(sv);
    s->launches++;
    rc = sp_check(s, "init");
    // the host tables go out of scope: wait for their copies
    if (rc == BL_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = sp_fail(s, BL_ECUDA, "init");
  } while (0);
  if (rc != BL_OK) {
    bl_sparse_destroy(s);
    return rc;
  }
  *out = s;
  return BL_OK;
}

extern "C" int bl_sparse_step(bl_sparse *s, int nsteps) {
  if (!s || nsteps < 0) return BL_EINVAL;
  if (s->sticky) return s->sticky;
  int k = 0;
  if (nsteps >= 2) {
    // pairs of steps as one graph launch (the graph starts at its parity)
    if (!s->gexec || s->g_parity != s->parity) {
      if (s->gexec) cudaGraphExecDestroy(s->gexec);
      s->gexec = nullptr;
      cudaGraph_t g = nullptr;
      SPCU(cudaStreamBeginCapture(s->gstream, cudaStreamCaptureModeThreadLocal));
      sp_launch_step(s, s->gstream, s->parity);
      sp_launch_step(s, s->gstream, s->parity ^ 1);
      SPCU(cudaStreamEndCapture(s->gstream, &g));
      const cudaError_t e = cudaGraphInstantiate(&s->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        s->gexec = nullptr;
        return sp_fail(s, BL_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
      }
      s->g_parity = s->parity;
    }
    SPCU(cudaEventRecord(s->ev_fork, s->stream));
    SPCU(cudaStreamWaitEvent(s->gstream, s->ev_fork, 0));
    for (; k + 2 <= nsteps; k += 2) {
      SPCU(cudaGraphLaunch(s->gexec, s->gstream));
      s->launches += 2;
    }
    SPCU(cudaEventRecord(s->ev_join, s->gstream));
    SPCU(cudaStreamWaitEvent(s->stream, s->ev_join, 0));
  }
  for (; k < nsteps; ++k) {
    sp_launch_step(s, s->stream, s->parity);
    s->parity ^= 1;
    s->launches++;
  }
  return sp_check(s, "step");
}

extern "C" int bl_sparse_sync(bl_sparse *s) {
  if (!s) return BL_EINVAL;
  const cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return sp_fail(s, BL_ECUDA, "stream: %s", cudaGetErrorString(e));
  if (s->sticky) return s->sticky;
  int st = 0;
  SPCU(cudaMemcpy(&st, s->sv.status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st & ST_UNSTABLE) return sp_fail(s, BL_EUNSTABLE, "unstable: rho <= 0, NaN or |u| >= 0.3 at some node");
  return BL_OK;
}

static int sp_scratch(bl_sparse *s, size_t bytes) {
  if (s->scratch_bytes >= bytes) return BL_OK;
  if (s->scratch) cudaFree(s->scratch);
  s->scratch = nullptr;
  s->scratch_bytes = 0;
  if (cudaMalloc(&s->scratch, bytes) != cudaSuccess) return sp_fail(s, BL_ENOMEM, "scratch");
  s->scratch_bytes = bytes;
  return BL_OK;
}

extern "C" int bl_sparse_fields_get(bl_sparse *s, double *rho, double *u, int on_device) {
  if (!s || (!rho && !u)) return BL_EINVAL;
  if (s->sticky) return s->sticky;
  const size_t N = (size_t)s->n_dense;
  double *dr = rho, *du = u;
  if (!on_device) {
    if (sp_scratch(s, sizeof(double) * 4 * N)) return s->sticky;
    dr = rho ? s->scratch : nullptr;
    du = u ? s->scratch + N : nullptr;
  }
  if (dr) SPCU(cudaMemsetAsync(dr, 0, sizeof(double) * N, s->stream));
  if (du) SPCU(cudaMemsetAsync(du, 0, sizeof(double) * 3 * N, s->stream));
  const unsigned b = 256, g = nblk(s->sv.Nf, b);
  if (s->lp.store_dtype == BL_STORE_F32) k_sparse_fields<float><<<g, b, 0, s->stream>>>(s->sv, s->parity, dr, du);
  else if (s->lp.store_dtype == BL_STORE_BF16) k_sparse_fields<__nv_bfloat16><<<g, b, 0, s->stream>>>(s->sv, s->parity, dr, du);
  else k_sparse_fields<__half><<<g, b, 0, s->stream>>>(s->sv, s->parity, dr, du);
  s->launches++;
  if (sp_check(s, "fields")) return s->sticky;
  if (!on_device) {
    if (rho) SPCU(cudaMemcpyAsync(rho, dr, sizeof(double) * N, cudaMemcpyDeviceToHost, s->stream));
    if (u) SPCU(cudaMemcpyAsync(u, du, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, s->stream));
  }
  return bl_sparse_sync(s);
}

static int sp_pop_io(bl_sparse *s, double *pop, int to_storage) {
  if (!s || !pop) return BL_EINVAL;
  if (s->sticky) return s->sticky;
  const size_t bytes = sizeof(double) * Q * (size_t)s->n_dense;
  if (sp_scratch(s, bytes)) return s->sticky;
  if (to_storage) SPCU(cudaMemcpyAsync(s->scratch, pop, bytes, cudaMemcpyHostToDevice, s->stream));
  else SPCU(cudaMemsetAsync(s->scratch, 0, bytes, s->stream));
  const unsigned b = 256, g = nblk(s->sv.Nf, b);
  if (s->lp.store_dtype == BL_STORE_F32) k_sparse_pop_io<float><<<g, b, 0, s->stream>>>(s->sv, s->parity, s->scratch, to_storage);
  else if (s->lp.store_dtype == BL_STORE_BF16)
    k_sparse_pop_io<__nv_bfloat16><<<g, b, 0, s->stream>>>(s->sv, s->parity, s->scratch, to_storage);
  else k_sparse_pop_io<__half><<<g, b, 0, s->stream>>>(s->sv, s->parity, s->scratch, to_storage);
  s->launches++;
  if (sp_check(s, "populations")) return s->sticky;
  if (!to_storage) SPCU(cudaMemcpyAsync(pop, s->scratch, bytes, cudaMemcpyDeviceToHost, s->stream));
  return bl_sparse_sync(s);
}

extern "C" int bl_sparse_populations_get(bl_sparse *s, double *pop) { return sp_pop_io(s, pop, 0); }

extern "C" int bl_sparse_populations_set(bl_sparse *s, const double *pop) {
  return sp_pop_io(s, const_cast<double *>(pop), 1);
}

extern "C" int bl_sparse_wall_momentum_get(bl_sparse *s, double *wallmom) {
  if (!s || !wallmom) return BL_EINVAL;
  if (s->sticky) return s->sticky;
  double F[NWALL * 3];
  long long K[NWALL * 3];
  SPCU(cudaMemcpyAsync(F, s->wa.F, sizeof(F), cudaMemcpyDeviceToHost, s->stream));
  SPCU(cudaMemcpyAsync(K, s->wa.K, sizeof(K), cudaMemcpyDeviceToHost, s->stream));
  SPCU(cudaStreamSynchronize(s->stream));
  SPCU(cudaMemsetAsync(s->wa.F, 0, sizeof(F), s->stream));
  SPCU(cudaMemsetAsync(s->wa.K, 0, sizeof(K), s->stream));
  for (int i = 0; i < NWALL * 3; ++i) wallmom[i] = F[i] + s->lp.rho0 / 18.0 * (double)K[i];
  return BL_OK;
}

extern "C" int64_t bl_sparse_nodes(const bl_sparse *s) { return s ? (int64_t)s->sv.Nf : -1; }

extern "C" int64_t bl_sparse_launch_count(const bl_sparse *s) { return s ? s->launches : -1; }

extern "C" const char *bl_sparse_last_error(const bl_sparse *s) { return s ? s->err : "null context"; }
