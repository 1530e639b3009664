// lb_sweep.cuh -- the lattice sweep of the coupled step (kernels and their
// launch for one storage type; lb_sweep_f32.cu, lb_sweep_bf16.cu and
// lb_sweep_f16.cu instantiate it, so that the three compile in parallel).
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
// yet (reading Q3, implicit coupling).  The node writes one link record per
// cell it borders (its direction mask, its density and, at tau = 1, its
// velocity moments, else the sum of 2 f~*_r c_r over those links) into the
// cell's bucket, from which the link kernel sums the cell's link momentum
// and drag matrices.  After the solve each node's record of its first cell
// becomes its pending velocity pu = rho (V + W x d) with the bounced
// directions; the next sweep reads pu with the populations and adds
// C = -(m_r / 6) c_r . pu (Eq. c, at the link midpoint; c_r . (W x c_r / 2)
// = 0) to those populations before the moments.  At tau = 1 the collision
// keeps only the moments of what it reads, so C enters as the change of
// rho and j it makes, summed over the bounced directions by popcount.
// Walls move at a known velocity: their links get C here, and the wall's
// momentum is summed per warp (constant part 2 alpha_r rho_bar c_r as exact
// integers) before one atomic per wall and component.
#pragma once

#include "bl_internal.cuh"

namespace bl {


// blocks of 128 threads resident per SM: 8 caps the per-thread copy
// pipeline at 64 registers
#ifndef BL_LB_MINB
#define BL_LB_MINB 8
#endif
// the one-node sweep: 9 blocks (56 registers, no spill at tau = 1) keep more
// loads in flight than 8 (64 registers): 94 -> 89.5 us at 128^3 with cells
#ifndef BL_ONE_MINB
#define BL_ONE_MINB 9
#endif
// the bulk-copy sweep: resident blocks per SM (its register cap) and stages
#ifndef BL_BULK_MINB
#define BL_BULK_MINB 6
#endif
#ifndef BL_BULK_TS
#define BL_BULK_TS 3
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

// the link records a node hands to the warp-level append: that of its first
// cell p (p < 0: no cell link) with its direction mask and the six values of
// the record, the density deviation drho and, at tau = 1, the node's u, uu
// and u . F, from which the link sums rebuild the bounced populations, else
// the sum of 2 f~*_r c_r over the mask (two zeros after it); and that of a
// second cell p2 (p2 < 0: none), with its own mask and, at tau != 1, its own
// sums f2 (at tau = 1 it shares the values)
struct CellLink {
  int p;
  uint32_t mask;
  float e[6];
  int p2;
  uint32_t mask2;
  float f2[3];
};

// warp-level append of the lanes' primary link records to their cells'
// buckets, one atomic per (warp, cell), in two halves so that the atomic's
// round trip can overlap other work (a block barrier): reserve takes the
// slots, write stores the records; all 32 lanes call both
struct LinkSlot {
  unsigned grp;
  int base;
};

__device__ __forceinline__ LinkSlot reserve_slots(const LatticeView &lv, int p) {
  const unsigned FULL = 0xffffffffu;
  LinkSlot sl{0u, 0};
  if (!__ballot_sync(FULL, p >= 0)) return sl;
  sl.grp = __match_any_sync(FULL, p);
  if (p >= 0 && (threadIdx.x & 31) == __ffs(sl.grp) - 1) sl.base = atomicAdd(&lv.rec_count[p], __popc(sl.grp));
  return sl;
}
__device__ __forceinline__ LinkSlot reserve_links(const LatticeView &lv, const CellLink &cl) {
  return reserve_slots(lv, cl.p);
}

__device__ __forceinline__ void write_links(const LatticeView &lv, const CellLink &cl, unsigned n, const LinkSlot &sl) {
  if (cl.p < 0) return;
  const int lane = threadIdx.x & 31;
  const int base = __shfl_sync(sl.grp, sl.base, __ffs(sl.grp) - 1);
  const int pos = base + __popc(sl.grp & ((1u << lane) - 1u));
  if (pos < lv.rec_cap) {
    float4 *r = lv.rec + 2 * ((size_t)cl.p * lv.rec_cap + pos);
    r[0] = make_float4(__uint_as_float(n), __uint_as_float(cl.mask), cl.e[0], cl.e[1]);
    r[1] = make_float4(cl.e[2], cl.e[3], cl.e[4], cl.e[5]);
  } else {
    atomicOr(lv.status, ST_OVERFLOW);
  }
}

// the second-cell record of this lane to its reserved slot, marked for C in
// place after the solve
template <bool TAU1>
__device__ __forceinline__ void write_second(const LatticeView &lv, const CellLink &cl, unsigned n,
                                             const LinkSlot &sl) {
  if (cl.p2 < 0) return;
  const int lane = threadIdx.x & 31;
  const int base = __shfl_sync(sl.grp, sl.base, __ffs(sl.grp) - 1);
  const int pos = base + __popc(sl.grp & ((1u << lane) - 1u));
  if (pos < lv.rec_cap) {
    float4 *r = lv.rec + 2 * ((size_t)cl.p2 * lv.rec_cap + pos);
    if constexpr (TAU1) {
      r[0] = make_float4(__uint_as_float(n), __uint_as_float(cl.mask2 | REC_DIRECT), cl.e[0], cl.e[1]);
      r[1] = make_float4(cl.e[2], cl.e[3], cl.e[4], cl.e[5]);
    } else {
      r[0] = make_float4(__uint_as_float(n), __uint_as_float(cl.mask2 | REC_DIRECT), cl.e[0], cl.f2[0]);
      r[1] = make_float4(cl.f2[1], cl.f2[2], 0.f, 0.f);
    }
  } else {
    atomicOr(lv.status, ST_OVERFLOW);
  }
}

// both records of the lanes (all 32 lanes call it): the two warp-level
// reservations in flight together, then the writes
template <bool TAU1>
__device__ __forceinline__ void emit_links(const LatticeView &lv, const CellLink &cl, unsigned n) {
  const LinkSlot sl = reserve_slots(lv, cl.p);
  const LinkSlot sl2 = reserve_slots(lv, cl.p2);
  write_links(lv, cl, n, sl);
  write_second<TAU1>(lv, cl, n, sl2);
}

// the second-cell records alone (kernels that write the first ones later)
template <bool TAU1>
__device__ __forceinline__ void emit_second(const LatticeView &lv, const CellLink &cl, unsigned n) {
  const LinkSlot sl2 = reserve_slots(lv, cl.p2);
  write_second<TAU1>(lv, cl, n, sl2);
}

// the neighbour n + c_r for a direction r known only at run time: the
// components of c_r + 1 from their packed form, the coordinate chosen by
// selects (no indexing of the xo, yo, zo arrays)
__device__ __forceinline__ unsigned pick3(unsigned k, const unsigned v[3]) { return k == 0 ? v[0] : (k == 1 ? v[1] : v[2]); }
__device__ __forceinline__ unsigned neighbour_rt(int r, const unsigned xo[3], const unsigned yo[3], const unsigned zo[3]) {
  constexpr unsigned long long PX = packed_dirs<0>(), PY = packed_dirs<1>(), PZ = packed_dirs<2>();
  return pick3((unsigned)(PX >> (2 * r)) & 3u, xo) + pick3((unsigned)(PY >> (2 * r)) & 3u, yo) +
         pick3((unsigned)(PZ >> (2 * r)) & 3u, zo);
}

// the pending C of the last step's bounces off a cell: pu.xyz = rho (V + W x
// d) of the cell at the node, pu.w the bounced directions (bit r); C_r =
// -(m_r / 6) c_r . pu is added to the incoming population of direction rbar
// (every direction computed, the masked ones kept: no branch per direction)
__device__ __forceinline__ void apply_pending(const float4 &pu, float (&f)[Q]) {
  using D = D3Q19;
  const uint32_t mask = __float_as_uint(pu.w);
  sfor<1, Q>([&](auto R) {
    constexpr int r = decltype(R)::value;
    float cu = 0.f;
    if constexpr (D::cx(r) != 0) cu += D::cx(r) * pu.x;
    if constexpr (D::cy(r) != 0) cu += D::cy(r) * pu.y;
    if constexpr (D::cz(r) != 0) cu += D::cz(r) * pu.z;
    f[D::opp(r)] -= ((mask >> r) & 1u) ? (D::m(r) / 6.0f) * cu : 0.0f;
  });
}

// the same C taken into the moments alone (enough at tau = 1, where the
// collision keeps nothing of a population but its moments):
// drho -= K . pu / 6, j += M pu / 6, K = sum m_r c_r, M = sum m_r c_r c_r^T
// over the bounced directions
__device__ __forceinline__ void pending_moments(const float4 &pu, float &drho, float &jx, float &jy, float &jz) {
  const uint32_t m = __float_as_uint(pu.w);
  const float s = 1.0f / 6.0f;
  drho -= s * ((float)mask_K<0>(m) * pu.x + (float)mask_K<1>(m) * pu.y + (float)mask_K<2>(m) * pu.z);
  const float mxy = (float)mask_Mab<0, 1>(m), mxz = (float)mask_Mab<0, 2>(m), myz = (float)mask_Mab<1, 2>(m);
  jx += s * ((float)mask_Maa<0>(m) * pu.x + mxy * pu.y + mxz * pu.z);
  jy += s * (mxy * pu.x + (float)mask_Maa<1>(m) * pu.y + myz * pu.z);
  jz += s * (mxz * pu.x + myz * pu.y + (float)mask_Maa<2>(m) * pu.z);
}

// sum of 2 f~*_r c_r over the directions in mask (no branch per direction)
__device__ __forceinline__ void link_sum(uint32_t mask, const float (&f)[Q], float (&F)[3]) {
  using D = D3Q19;
  float F0 = 0.f, F1 = 0.f, F2 = 0.f;
  sfor<1, Q>([&](auto R) {
    constexpr int r = decltype(R)::value;
    const float v = ((mask >> r) & 1u) ? 2.0f * f[r] : 0.0f;
    if constexpr (D::cx(r) != 0) F0 += D::cx(r) * v;
    if constexpr (D::cy(r) != 0) F1 += D::cy(r) * v;
    if constexpr (D::cz(r) != 0) F2 += D::cz(r) * v;
  });
  F[0] = F0;
  F[1] = F1;
  F[2] = F2;
}

// one record appended to cell q's bucket by this thread alone
__device__ __forceinline__ void append_link(const LatticeView &lv, unsigned n, int q, uint32_t mask,
                                            const float (&e)[6]) {
  const int pos = atomicAdd(&lv.rec_count[q], 1);
  if (pos < lv.rec_cap) {
    float4 *rr = lv.rec + 2 * ((size_t)q * lv.rec_cap + pos);
    rr[0] = make_float4(__uint_as_float(n), __uint_as_float(mask), e[0], e[1]);
    rr[1] = make_float4(e[2], e[3], e[4], e[5]);
  } else {
    atomicOr(lv.status, ST_OVERFLOW);
  }
}

// One fluid node of the sweep: the pending C of its last bounces off a cell,
// moments, collision, streaming with bounce-back, the wall momentum and its
// cell links.  load(r, slot) gives the incoming population of direction r
// (from the slot src_slot names); pu is the node's pending velocity.
// FORCE: a body force is set (Guo forcing); TAU1: tau = 1, where the
// relaxation gives the equilibrium itself
template <class S, int PAR, bool FORCE, bool TAU1, class Load>
__device__ __forceinline__ void node_update(const LatticeView &lv, const WallAcc &wa, unsigned n, const int xyz[3],
                                            const unsigned xo[3], const unsigned yo[3], const unsigned zo[3],
                                            uint32_t nbw, uint32_t nbc, float4 pu, Load load, int &wkey,
                                            float (&wF)[3], int (&wK)[3], CellLink &cl) {
  using D = D3Q19;
  const unsigned N = lv.N;
  S *pop = reinterpret_cast<S *>(lv.pop);
  cl.p = -1;
  cl.p2 = -1;
  if (nbw & NB_FLUID) {
    const unsigned solid = nbw & NB_SOLID;
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
    // C of the last step's bounces off a cell (reading Q3): into the
    // populations, or at tau = 1 into the moments
    const uint32_t pm = __float_as_uint(pu.w);
    if constexpr (!TAU1) {
      if (pm) apply_pending(pu, f);
    }
    // moments (shifted: rho = rho_bar + sum f~, j = sum f~ c)
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
    sfor<0, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      drho += f[r];
      if constexpr (D::cx(r) != 0) jx += D::cx(r) * f[r];
      if constexpr (D::cy(r) != 0) jy += D::cy(r) * f[r];
      if constexpr (D::cz(r) != 0) jz += D::cz(r) * f[r];
    });
    if constexpr (TAU1) {
      if (pm) pending_moments(pu, drho, jx, jy, jz);
    }
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
    if (!(rho > 0.f) || !(uu < 0.09f)) atomicOr(lv.status, ST_UNSTABLE);
    // the moments of the nodes beside a sheared plane, for its passes
    if (lv.le_mom != nullptr && (xyz[0] == 0 || xyz[0] == lv.nx - 1))
      lv.le_mom[(xyz[0] == 0 ? 0u : (unsigned)lv.ny * (unsigned)lv.nz) + (unsigned)xyz[1] +
                (unsigned)lv.ny * (unsigned)xyz[2]] = make_float4(drho, ux, uy, uz);
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
    // neighbour classes from the geometry pass: solid = any non-fluid node;
    // next to a wall or a cell the owners of the solid neighbours give the
    // walls and the cells (in direction order: the first and a second cell
    // each get a record and a pending C; a third, rare, its links one by one)
    if (nbw & (NB_WALL | NB_CELL)) {
      unsigned wall = 0, cmask = 0, cmask2 = 0, csec = 0;
      int p1 = -1, p2 = -1;
      // one cell and nothing else next to the node (the common case): its
      // index from the neighbour-cell word, no owner to read
      const bool one_cell = !(nbc & NBC_MIXED);
      if (one_cell) {
        p1 = (int)nbc;
        cmask = solid;
      }
      for (unsigned m = one_cell ? 0u : solid; m; m &= m - 1u) {
        const int r = __ffs(m) - 1;
        const int ow = lv.owner[neighbour_rt(r, xo, yo, zo)];
        if (ow <= -2) {
          wall |= 1u << r;
        } else if (p1 < 0 || ow == p1) {
          p1 = ow;
          cmask |= 1u << r;
        } else if (p2 < 0 || ow == p2) {
          p2 = ow;
          cmask2 |= 1u << r;
        } else {
          csec |= 1u << r;
        }
      }
      if (wall) {
        // links into a wall: the moving-wall term C for the population
        // returning along rbar, 6 alpha_rbar rho c_rbar . v_wall, and the
        // momentum the wall receives
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
      // cell links: the record of the first cell through the warp-level
      // append; those of a second and a third cell, rarer, directly, marked
      // for C in place after the solve.  At tau = 1 a record holds the
      // node's moments (the same for every cell of the node), else the sum
      // of 2 f~*_r c_r over its directions
      if (cmask) {
        cl.p = p1;
        cl.mask = cmask;
        cl.e[0] = drho;
        if constexpr (TAU1) {
          cl.e[1] = ux;
          cl.e[2] = uy;
          cl.e[3] = uz;
          cl.e[4] = uu;
          cl.e[5] = uF;
        } else {
          float F[3];
          link_sum(cmask, f, F);
          cl.e[1] = F[0];
          cl.e[2] = F[1];
          cl.e[3] = F[2];
          cl.e[4] = cl.e[5] = 0.f;
        }
        if (cmask2) {
          cl.p2 = p2;
          cl.mask2 = cmask2;
          if constexpr (!TAU1) link_sum(cmask2, f, cl.f2);
        }
        if (csec) {
          sfor<1, Q>([&](auto R) {
            constexpr int r = decltype(R)::value;
            if (csec & (1u << r)) {
              const unsigned nb = xo[1 + D::cx(r)] + yo[1 + D::cy(r)] + zo[1 + D::cz(r)];
              float e[6] = {drho, cl.e[1], cl.e[2], cl.e[3], cl.e[4], cl.e[5]};
              if constexpr (!TAU1) {
                e[1] = 2.0f * D::cx(r) * f[r];
                e[2] = 2.0f * D::cy(r) * f[r];
                e[3] = 2.0f * D::cz(r) * f[r];
              }
              append_link(lv, n, lv.owner[nb], (1u << r) | REC_DIRECT, e);
            }
          });
        }
      }
    }
    // a node whose C was pending and that has no first-cell record now: no
    // pending C for the next sweep (a record's pu is written after the solve)
    if (pm && cl.p < 0) reinterpret_cast<float *>(lv.pu + n)[3] = 0.f;
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
  }
}

template <class S, int PAR, bool FORCE, bool TAU1>
__global__ void __launch_bounds__(128, BL_ONE_MINB) k_lb_step(LatticeView lv, WallAcc wa) {
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
  // the node's populations, neighbour-cell word and pending velocity are
  // requested with its neighbour word, before it is known whether the node
  // is fluid: one memory round trip per node instead of two (a solid node's
  // values are discarded; every slot read lies in the population array)
  float fin[Q];
  uint32_t nbcv = NBC_MIXED;
  float4 puv = make_float4(0.f, 0.f, 0.f, 0.f);
  if (valid) {
    sfor<0, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      fin[r] = Store<S>::ld(pop + src_slot<PAR>(r, lv.N, n, xo, yo, zo));
    });
    nbcv = lv.nbc[n];
    puv = lv.pu[n];
  }
  // wall momentum of this thread: wall id, variable part, constant-part integers
  int wkey = -1;
  float wF[3] = {0.f, 0.f, 0.f};
  int wK[3] = {0, 0, 0};
  CellLink cl;
  cl.p = -1;
  cl.p2 = -1;
  if (nbw & NB_FLUID) {
    const int xyz[3] = {x, y, z};
    node_update<S, PAR, FORCE, TAU1>(lv, wa, n, xyz, xo, yo, zo, nbw, nbcv, puv,
                                     [&](int r, unsigned) { return fin[r]; }, wkey, wF, wK, cl);
  }
  emit_links<TAU1>(lv, cl, n);
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
__global__ void __launch_bounds__(128, BL_LB_MINB) k_lb_step_pipe(LatticeView lv, WallAcc wa) {
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
    CellLink cl;
    cl.p = -1;
    cl.p2 = -1;
    unsigned zo[3];
    zoff(z, zo);
    if (w[0] & NB_FLUID) {
      const int xyz[3] = {x, y, z};
      node_update<float, PAR, FORCE, TAU1>(lv, wa, rowb + zo[1], xyz, xo, yo, zo, w[0], lv.nbc[rowb + zo[1]],
                                           lv.pu[rowb + zo[1]],
                                           [&](int r, unsigned) { return stage[b][r][tx]; }, wkey, wF, wK, cl);
    }
    emit_links<TAU1>(lv, cl, rowb + zo[1]);
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
__global__ void __launch_bounds__(128, BL_BULK_MINB) k_lb_step_bulk(LatticeView lv, WallAcc wa) {
  using D = D3Q19;
  __shared__ alignas(128) S sb[TS][Q][128];        // [stage][array][x]
  __shared__ alignas(128) uint32_t sw[TS][128];    // [stage][x] neighbour words
  __shared__ alignas(128) float4 spu[TS][128];     // [stage][x] pending velocities
  __shared__ alignas(128) uint32_t sc[TS][128];    // [stage][x] neighbour-cell words
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
    mbar_expect_tx(&bar[s], Q * bytes + (unsigned)W * 24u);
    sfor<0, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      unsigned row;
      if constexpr (PAR == 0 || r == 0) row = (unsigned)r * N + yo[1] + zo[1];
      else row = (unsigned)D::opp(r) * N + yo[1 - D::cy(r)] + zo[1 - D::cz(r)];
      bulk_g2s(&sb[s][r][0], pop + row + (unsigned)x0, bytes, &bar[s]);
    });
    bulk_g2s(&sw[s][0], lv.nbm + yo[1] + zo[1] + (unsigned)x0, (unsigned)W * 4u, &bar[s]);
    bulk_g2s(&spu[s][0], lv.pu + yo[1] + zo[1] + (unsigned)x0, (unsigned)W * 16u, &bar[s]);
    bulk_g2s(&sc[s][0], lv.nbc + yo[1] + zo[1] + (unsigned)x0, (unsigned)W * 4u, &bar[s]);
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
      atomicOr(lv.status, ST_BARRIER);
      s_ok = 0;
    }
    __syncthreads();
    if (!s_ok) break;
    const uint32_t w = valid ? sw[s][tx] : 0u;
    unsigned zo[3];
    zoff(z, zo);
    const unsigned n = (unsigned)x + yo[1] + zo[1];
    CellLink cl;
    cl.p = -1;
    cl.p2 = -1;
    if (w & NB_FLUID) {
      const int xyz[3] = {x, y, z};
      node_update<S, PAR, FORCE, TAU1>(
          lv, wa, n, xyz, xo, yo, zo, w, sc[s][tx], spu[s][tx],
          [&](int r, unsigned slot) -> float {
            if (PAR == 0 || r == 0) return Store<S>::ld(&sb[s][r][tx]);
            int j = tx - D::cx(r);
            if (whole) j = j < 0 ? j + W : (j >= W ? j - W : j);
            return (j >= 0 && j < W) ? Store<S>::ld(&sb[s][r][j]) : Store<S>::ld(pop + slot);
          },
          wkey, wF, wK, cl);
    }
    const LinkSlot sl = reserve_links(lv, cl);
    const LinkSlot sl2 = reserve_slots(lv, cl.p2);
    __syncthreads();  // stage s is read: free for refill (the atomics' round trip overlaps it)
    write_links(lv, cl, n, sl);
    write_second<TAU1>(lv, cl, n, sl2);
  }
  if (z < ze && tx == 0) {
    // gave up: let the copies still in flight land before the block exits
    for (int k = 0; k < TS; ++k) mbar_wait(&bar[k], 0u), mbar_wait(&bar[k], 1u);
  }
  flush_wall_momentum(wa, wkey, wF, wK);
}

// ---------------------------------------------------------------------------
// host-side launch of the sweep

template <int PAR, bool FORCE, bool TAU1, int ZC>
static void launch_pipe(const LatticeView &lv, dim3 grid, dim3 block, const WallAcc &wa, cudaStream_t st) {
  const dim3 gp(grid.x, grid.y, (grid.z + ZC - 1) / ZC);
  k_lb_step_pipe<PAR, FORCE, TAU1, ZC><<<gp, block, 0, st>>>(lv, wa);
}

template <class S, int PAR, bool FORCE, bool TAU1, int ZC, int TS>
static void launch_bulk(const LatticeView &lv, dim3 grid, const WallAcc &wa, cudaStream_t st) {
  const dim3 gp((lv.nx + 127) / 128, grid.y, (grid.z + ZC - 1) / ZC);
  k_lb_step_bulk<S, PAR, FORCE, TAU1, ZC, TS><<<gp, 128, 0, st>>>(lv, wa);
}

// The persistent row sweep: a grid of as many blocks as the device holds at
// once, block b taking the rows (segment, y, z) numbered b, b + G, b + 2G,
// ... (G blocks, segments of 128 nodes fastest) in one bulk-copy pipeline
// TS - 1 rows ahead, so that no tail wave and no pipeline restart remain.
// The link records of a row wait in shared memory until the next row is
// collided, by when the bucket atomic that gave them their slots has
// returned; one barrier per row frees its stage.  Row and wait rules as in
// k_lb_step_bulk.
#ifndef BL_ROWS_MINB
#define BL_ROWS_MINB 5
#endif
#ifndef BL_ROWS_TS
#define BL_ROWS_TS 3
#endif

struct RowGeo {
  int x0, W, y, z;
};

// the staged record of this lane, written to the slot reserved one row before
__device__ __forceinline__ void write_staged(const LatticeView &lv, int p, unsigned grp, int base0, const float4 &r0,
                                             const float4 &r1) {
  if (p < 0) return;
  const int lane = threadIdx.x & 31;
  const int base = __shfl_sync(grp, base0, __ffs(grp) - 1);
  const int pos = base + __popc(grp & ((1u << lane) - 1u));
  if (pos < lv.rec_cap) {
    float4 *r = lv.rec + 2 * ((size_t)p * lv.rec_cap + pos);
    r[0] = r0;
    r[1] = r1;
  } else {
    atomicOr(lv.status, ST_OVERFLOW);
  }
}

template <class S, int PAR, bool FORCE, bool TAU1, int TS>
__global__ void __launch_bounds__(128, BL_ROWS_MINB) k_lb_step_rows(LatticeView lv, WallAcc wa) {
  using D = D3Q19;
  __shared__ alignas(128) S sb[TS][Q][128];      // [stage][array][x]
  __shared__ alignas(128) uint32_t sw[TS][128];  // [stage][x] neighbour words
  __shared__ alignas(128) float4 spu[TS][128];   // [stage][x] pending velocities
  __shared__ alignas(128) uint32_t sc[TS][128];  // [stage][x] neighbour-cell words
  __shared__ alignas(128) float4 srec[2][128];   // the last row's link record of each thread
  __shared__ alignas(8) unsigned long long bar[TS];
  const int nx = lv.nx, ny = lv.ny, nz = lv.nz;
  const int tx = threadIdx.x;
  const int nseg = (nx + 127) >> 7;
  const int nitems = nseg * ny * nz;
  const int G = gridDim.x;
  const int kmax = (int)blockIdx.x < nitems ? (nitems - 1 - (int)blockIdx.x) / G + 1 : 0;
  const unsigned N = lv.N;
  const unsigned nxy = (unsigned)nx * (unsigned)ny;
  const S *pop = reinterpret_cast<const S *>(lv.pop);
  auto geo = [&](int k) {
    const int it = (int)blockIdx.x + k * G;
    const int seg = it % nseg, t = it / nseg;
    RowGeo g;
    g.x0 = seg << 7;
    g.W = min(128, nx - g.x0);
    g.y = t % ny;
    g.z = t / ny;
    return g;
  };
  auto yzo = [&](const RowGeo &g, unsigned yo[3], unsigned zo[3]) {
    yo[0] = (unsigned)(g.y == 0 ? ny - 1 : g.y - 1) * nx;
    yo[1] = (unsigned)g.y * nx;
    yo[2] = (unsigned)(g.y == ny - 1 ? 0 : g.y + 1) * nx;
    zo[0] = (unsigned)(g.z == 0 ? nz - 1 : g.z - 1) * nxy;
    zo[1] = (unsigned)g.z * nxy;
    zo[2] = (unsigned)(g.z == nz - 1 ? 0 : g.z + 1) * nxy;
  };
  // one thread: the copies of row k into stage s
  auto issue = [&](int k, int s) {
    const RowGeo g = geo(k);
    unsigned yo[3], zo[3];
    yzo(g, yo, zo);
    const unsigned bytes = (unsigned)g.W * (unsigned)sizeof(S);
    mbar_expect_tx(&bar[s], Q * bytes + (unsigned)g.W * 24u);
    sfor<0, Q>([&](auto R) {
      constexpr int r = decltype(R)::value;
      unsigned row;
      if constexpr (PAR == 0 || r == 0) row = (unsigned)r * N + yo[1] + zo[1];
      else row = (unsigned)D::opp(r) * N + yo[1 - D::cy(r)] + zo[1 - D::cz(r)];
      bulk_g2s(&sb[s][r][0], pop + row + (unsigned)g.x0, bytes, &bar[s]);
    });
    const unsigned o = yo[1] + zo[1] + (unsigned)g.x0;
    bulk_g2s(&sw[s][0], lv.nbm + o, (unsigned)g.W * 4u, &bar[s]);
    bulk_g2s(&spu[s][0], lv.pu + o, (unsigned)g.W * 16u, &bar[s]);
    bulk_g2s(&sc[s][0], lv.nbc + o, (unsigned)g.W * 4u, &bar[s]);
  };
  if (tx == 0) {
    for (int k = 0; k < TS; ++k) mbar_init(&bar[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (tx == 0)
    for (int k = 0; k < TS - 1 && k < kmax; ++k) issue(k, k);
  int wkey = -1;
  float wF[3] = {0.f, 0.f, 0.f};
  int wK[3] = {0, 0, 0};
  // the slot of this thread's record of the last row: cell, lane group, base
  int lp = -1;
  unsigned lgrp = 0u;
  int lbase = 0;
  bool failed = false;
  for (int k = 0; k < kmax; ++k) {
    const int s = k % TS;
    if (tx == 0 && k + TS - 1 < kmax) issue(k + TS - 1, (k + TS - 1) % TS);  // freed by the last barrier
    const bool ok = mbar_wait(&bar[s], (unsigned)(k / TS) & 1u);
    if (!ok) atomicOr(lv.status, ST_BARRIER);
    const RowGeo g = geo(k);
    const bool whole = g.W == nx;
    const bool valid = tx < g.W;
    const int x = g.x0 + (valid ? tx : g.W - 1);
    const unsigned xo[3] = {(unsigned)(x == 0 ? nx - 1 : x - 1), (unsigned)x, (unsigned)(x == nx - 1 ? 0 : x + 1)};
    unsigned yo[3], zo[3];
    yzo(g, yo, zo);
    const uint32_t w = (valid && ok) ? sw[s][tx] : 0u;
    const unsigned n = (unsigned)x + yo[1] + zo[1];
    CellLink cl;
    cl.p = -1;
    cl.p2 = -1;
    if (w & NB_FLUID) {
      const int xyz[3] = {x, g.y, g.z};
      const int W = g.W;
      node_update<S, PAR, FORCE, TAU1>(
          lv, wa, n, xyz, xo, yo, zo, w, sc[s][tx], spu[s][tx],
          [&](int r, unsigned slot) -> float {
            if (PAR == 0 || r == 0) return Store<S>::ld(&sb[s][r][tx]);
            int j = tx - D::cx(r);
            if (whole) j = j < 0 ? j + W : (j >= W ? j - W : j);
            return (j >= 0 && j < W) ? Store<S>::ld(&sb[s][r][j]) : Store<S>::ld(pop + slot);
          },
          wkey, wF, wK, cl);
    }
    // the last row's records to the slots reserved then; this row's slots
    // reserved now, its records staged
    write_staged(lv, lp, lgrp, lbase, srec[0][tx], srec[1][tx]);
    emit_second<TAU1>(lv, cl, n);
    const LinkSlot sl = reserve_links(lv, cl);
    if (cl.p >= 0) {
      srec[0][tx] = make_float4(__uint_as_float(n), __uint_as_float(cl.mask), cl.e[0], cl.e[1]);
      srec[1][tx] = make_float4(cl.e[2], cl.e[3], cl.e[4], cl.e[5]);
    }
    lp = cl.p;
    lgrp = sl.grp;
    lbase = sl.base;
    if (__syncthreads_or(!ok)) {  // stage s is read: free for refill
      failed = true;
      break;
    }
  }
  write_staged(lv, lp, lgrp, lbase, srec[0][tx], srec[1][tx]);
  if (failed && tx == 0) {
    // gave up: let the copies still in flight land before the block exits
    for (int k = 0; k < TS; ++k) mbar_wait(&bar[k], 0u), mbar_wait(&bar[k], 1u);
  }
  flush_wall_momentum(wa, wkey, wF, wK);
}

template <class S, int PAR, bool FORCE, bool TAU1>
static void launch_rows(const LatticeView &lv, const WallAcc &wa, cudaStream_t st) {
  const int nitems = ((lv.nx + 127) / 128) * lv.ny * lv.nz;
  const int g = lv.rows_grid[PAR * 4 + (FORCE ? 2 : 0) + (TAU1 ? 1 : 0)];
  k_lb_step_rows<S, PAR, FORCE, TAU1, BL_ROWS_TS><<<min(g > 0 ? g : 1, nitems), 128, 0, st>>>(lv, wa);
}

// the persistent sweep's grid for each instantiation (index PAR * 4 + FORCE
// * 2 + TAU1): SMs x resident blocks per SM
template <class S>
static void rows_grids(int out[8]) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void *k[8] = {(const void *)k_lb_step_rows<S, 0, false, false, BL_ROWS_TS>,
                      (const void *)k_lb_step_rows<S, 0, false, true, BL_ROWS_TS>,
                      (const void *)k_lb_step_rows<S, 0, true, false, BL_ROWS_TS>,
                      (const void *)k_lb_step_rows<S, 0, true, true, BL_ROWS_TS>,
                      (const void *)k_lb_step_rows<S, 1, false, false, BL_ROWS_TS>,
                      (const void *)k_lb_step_rows<S, 1, false, true, BL_ROWS_TS>,
                      (const void *)k_lb_step_rows<S, 1, true, false, BL_ROWS_TS>,
                      (const void *)k_lb_step_rows<S, 1, true, true, BL_ROWS_TS>};
  for (int i = 0; i < 8; ++i) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k[i], 128, 0) != cudaSuccess || b < 1) b = 1;
    out[i] = (sms > 0 ? sms : 1) * b;
  }
}

// row length for the bulk-copy sweep: 16-byte aligned rows of the storage type
__host__ __device__ inline bool bulk_rows_ok(int nx, int store_bytes) { return nx % (16 / store_bytes) == 0; }

// sweep variants (LatticeView::sweep): 0 one node per thread; 1, 2 the FP32
// pipeline over 4 or 8 planes; 3, 4 the bulk-copy pipeline over 8 or 4 planes
// with 3 stages; 5 the persistent bulk-copy row sweep (3 to 5: any storage
// type with 16-byte aligned rows, else variant 0)
template <class S, int PAR, bool FORCE, bool TAU1>
static void launch_lb_variant(const LatticeView &lv, dim3 grid, dim3 block, const WallAcc &wa, cudaStream_t st) {
  if constexpr (std::is_same<S, float>::value) {
    if (lv.sweep == 1) return launch_pipe<PAR, FORCE, TAU1, 4>(lv, grid, block, wa, st);
    if (lv.sweep == 2) return launch_pipe<PAR, FORCE, TAU1, 8>(lv, grid, block, wa, st);
  }
  if (bulk_rows_ok(lv.nx, (int)sizeof(S))) {
    if (lv.sweep == 3) return launch_bulk<S, PAR, FORCE, TAU1, 8, BL_BULK_TS>(lv, grid, wa, st);
    if (lv.sweep == 4) return launch_bulk<S, PAR, FORCE, TAU1, 4, BL_BULK_TS>(lv, grid, wa, st);
    if (lv.sweep == 5) return launch_rows<S, PAR, FORCE, TAU1>(lv, wa, st);
  }
  k_lb_step<S, PAR, FORCE, TAU1><<<grid, block, 0, st>>>(lv, wa);
}

template <class S, int PAR, bool FORCE>
static void launch_lb_tau(const LatticeView &lv, dim3 grid, dim3 block, const WallAcc &wa, cudaStream_t st) {
  if (lv.omega == 1.0f) launch_lb_variant<S, PAR, FORCE, true>(lv, grid, block, wa, st);
  else launch_lb_variant<S, PAR, FORCE, false>(lv, grid, block, wa, st);
}

template <class S>
static void launch_lb_typed(const LatticeView &lv, int par, const WallAcc &wa, cudaStream_t st) {
  const int bx = lv.nx >= 128 ? 128 : ((lv.nx + 31) / 32) * 32;
  dim3 block(bx, 1, 1);
  dim3 grid((lv.nx + bx - 1) / bx, lv.ny, lv.nz);
  if (par == 0) {
    if (lv.has_force) launch_lb_tau<S, 0, true>(lv, grid, block, wa, st);
    else launch_lb_tau<S, 0, false>(lv, grid, block, wa, st);
  } else {
    if (lv.has_force) launch_lb_tau<S, 1, true>(lv, grid, block, wa, st);
    else launch_lb_tau<S, 1, false>(lv, grid, block, wa, st);
  }
}

}  // namespace bl
