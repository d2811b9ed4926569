// Team-cooperative executor: the tier for large classes (FusionRCG Sec.
// III-C, Regime II, re-derived for GB300).
//
// A team of T lanes (T = 32 to 512; one to sixteen warps) evaluates one
// shell quartet: it walks the quartet's primitive quartets one at a time
// (Algorithm 2's loops, accumulate-then-transform), and for each it runs the
// Phase-1 graph wave by wave -- a wave is a set of mutually independent nodes
// in DSA order (Eq. 7), cut into steps of ILP nodes per lane -- with a team
// barrier between waves.  Phase 2 (HRR + stepwise transform, Eq. 16) and the
// output stores run the same way once per shell quartet.
//
// The value slots of one primitive quartet are shared by the whole team, so
// a class whose live set is thousands of values stays in shared memory; the
// accumulator bank H sits in shared memory when it fits, else in a
// team-private global region (L2-resident).  Operand ids: id < nh is H[id],
// id >= nh is value slot id - nh; slots beyond the shared-memory part spill to
// a team-private global region.
#include <algorithm>

#include "eri_common.cuh"
#include "eri_coop.cuh"


__device__ __forceinline__ double eri_coop_pick8(int k, const double (&t)[8]) {
  double r = t[0];
#pragma unroll
  for (int i = 1; i < 8; ++i) r = (k == i + 1) ? t[i] : r;
  return r;
}

__device__ __forceinline__ double eri_coop_pick3(int i, double x, double y, double z) {
  return i == 0 ? x : (i == 1 ? y : z);
}

__device__ __forceinline__ void eri_coop_boys(int L, double T, double* F, const double* __restrict__ tab) {
  const double ex = exp(-T);
  if (T < ERI_BOYS_TMAX) {
    const int k = __double2int_rn(T * ERI_BOYS_INV_STEP);
    const double d = T - k * ERI_BOYS_STEP;
    const double* r = tab + k * ERI_BOYS_NCOL + L;
    double acc = __ldg(r + ERI_BOYS_NTAY - 1);
#pragma unroll
    for (int j = ERI_BOYS_NTAY - 1; j >= 1; --j) acc = fma(acc, -d * (1.0 / j), __ldg(r + j - 1));
    F[L] = acc;
    for (int m = L - 1; m >= 0; --m) F[m] = fma(2.0 * T, F[m + 1], ex) * eri_inv_odd[m];
  } else {
    const double rt = rsqrt(T);
    F[0] = 0.88622692545275801365 * rt;
    const double h = 0.5 * rt * rt;
    for (int m = 0; m < L; ++m) F[m + 1] = fma((double)(2 * m + 1), F[m], -ex) * h;
  }
}

// Per-primitive-quartet coefficient row, computed by one lane for a batch of
// primitive quartets and then read by the whole team:
//   [0, 17)   base values pref * F_m(T), m = 0..16
//   17 + 6 side + 3 j + axis   (P-A | W-P) for side 0, (Q-C | W-Q) for side 1
//   29 + 8 side + k - 1        k / (2 zeta) (side 0), k / (2 eta) (side 1)
//   45 + k - 1                 k / (2 (zeta + eta))
//   53 + side                  -rho/zeta, -rho/eta
#define ERI_COOP_NC 56
#define ERI_COOP_BATCH 32  // largest row batch (one row per lane of a warp)

// The FP64 row (value type R = double).
template <typename R>
__device__ __forceinline__ void eri_coop_row(const EriPairPrim& bp, const EriPairPrim& kp, int L,
                                             const double* __restrict__ tab, R* row) {
  EriPrimQuartet pq;
  eri_prim_quartet(bp, kp, pq);
  double F[ERI_BOYS_LMAX + 1];
  eri_coop_boys(L, pq.T, F, tab);
  for (int m = 0; m <= L; ++m) row[m] = (R)(pq.pref * F[m]);
  for (int i = 0; i < 3; ++i) {
    row[17 + i] = (R)bp.PA[i];
    row[20 + i] = (R)pq.WP[i];
    row[23 + i] = (R)kp.PA[i];
    row[26 + i] = (R)pq.WQ[i];
  }
  for (int k = 0; k < 8; ++k) {
    row[29 + k] = (R)((double)(k + 1) * bp.inv2z);
    row[37 + k] = (R)((double)(k + 1) * kp.inv2z);
    row[45 + k] = (R)((double)(k + 1) * (0.5 * pq.s));
  }
  row[53] = (R)(-pq.te);
  row[54] = (R)(-pq.tz);
}

// The FP32 row of a quartet whose recurrences run in FP32: formed in FP32
// from the FP32 pair data, with the Boys function in FP64.
__device__ __forceinline__ void eri_coop_row(const EriPairPrimF& bp, const EriPairPrimF& kp, int L,
                                             const double* __restrict__ tab, float* row) {
  EriPrimQuartetF pq;
  eri_prim_quartet_f32(bp, kp, pq);
  double F[ERI_BOYS_LMAX + 1];
  eri_coop_boys(L, (double)pq.T, F, tab);
  for (int m = 0; m <= L; ++m) row[m] = pq.pref * (float)F[m];
  for (int i = 0; i < 3; ++i) {
    row[17 + i] = bp.PA[i];
    row[20 + i] = pq.WP[i];
    row[23 + i] = kp.PA[i];
    row[26 + i] = pq.WQ[i];
  }
  const float c3 = 0.5f * pq.s;
  for (int k = 0; k < 8; ++k) {
    row[29 + k] = (float)(k + 1) * bp.inv2z;
    row[37 + k] = (float)(k + 1) * kp.inv2z;
    row[45 + k] = (float)(k + 1) * c3;
  }
  row[53] = -pq.te;
  row[54] = -pq.tz;
}

// The primitive-pair records a team of value type R forms its rows from.
template <typename R>
struct EriPrimsOf {
  static __device__ __forceinline__ const EriPairPrim* get(const EriLaunchArgs& a) { return a.pprims; }
};
template <>
struct EriPrimsOf<float> {
  static __device__ __forceinline__ const EriPairPrimF* get(const EriLaunchArgs& a) { return a.pprims_f; }
};

__device__ __forceinline__ double eri_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float eri_fma(float a, float b, float c) { return fmaf(a, b, c); }

// Phase-1 nodes (descriptor: see the generator's coop module).  Operands
// are value slots in the team's shared memory; a lane's two nodes of a step
// belong to one wave and never alias, so both nodes' operands are loaded
// before either result is stored and the two FMA chains interleave.
template <typename R>
struct EriCoopOps {
  R a, b, c, d, e;
};

template <typename R>
__device__ __forceinline__ void eri_coop_load1(const uint4& d, const R* V, EriCoopOps<R>& v) {
  const unsigned meta = d.w >> 16;
  if (meta & 0xC000u) return;  // no-op or base node
  v.a = V[d.y & 0xFFFF];
  v.b = V[d.y >> 16];
  if (meta & (31u << 4)) {
    v.c = V[d.z & 0xFFFF];
    v.d = V[d.z >> 16];
  }
  if (meta & (15u << 9)) v.e = V[d.w & 0xFFFF];
}

// Every lane of the warp calls this (no-op lanes included).  A warp issues
// an FP64 instruction when any of its lanes executes it.  VOTE: each
// optional part of the node sits behind a warp vote, so a warp none of whose
// lanes needs it skips it (lanes are packed by node shape, so most warps
// agree); else the parts are predicated per lane and the compiler decides.
template <bool VOTE, typename R>
__device__ __forceinline__ R eri_coop_eval1(const uint4& d, const R* row, const EriCoopOps<R>& v) {
  const unsigned meta = d.w >> 16;
  const unsigned k = (meta >> 4) & 31;
  if (!VOTE) {
    if (meta & 0x4000u) return row[k];  // base node: pref * F_m
    const unsigned cgo = meta & 15, k3 = (meta >> 9) & 15, side = (meta >> 13) & 1;
    R x = row[17 + cgo] * v.a;
    x = eri_fma(row[20 + cgo], v.b, x);
    if (k) x = eri_fma(row[28 + 8 * side + k], eri_fma(row[53 + side], v.d, v.c), x);
    if (k3) x = eri_fma(row[44 + k3], v.e, x);
    return x;
  }
  const bool term = (meta & 0xC000u) == 0;
  const bool t2 = term && k != 0, t3 = term && (meta & (15u << 9)) != 0;
  R x = (meta & 0x4000u) ? row[k] : (R)0;  // base node: pref * F_m
  if (__any_sync(0xffffffffu, term)) {
    const unsigned cgo = meta & 15;
    if (term) {
      x = row[17 + cgo] * v.a;
      x = eri_fma(row[20 + cgo], v.b, x);
    }
  }
  if (__any_sync(0xffffffffu, t2)) {
    const unsigned side = (meta >> 13) & 1;
    if (t2) x = eri_fma(row[28 + 8 * side + k], eri_fma(row[53 + side], v.d, v.c), x);
  }
  if (__any_sync(0xffffffffu, t3)) {
    const unsigned k3 = (meta >> 9) & 15;
    if (t3) x = eri_fma(row[44 + k3], v.e, x);
  }
  return x;
}

template <bool HSM, typename R>
__device__ __forceinline__ void eri_coop_store1(const uint4& d, R x, R* V, R* H) {
  if ((d.w >> 16) & 0x8000u) return;
  const unsigned dst = d.x & 0xFFFF, h = d.x >> 16;
  if (dst != 0xFFFF) V[dst] = x;
  if (h) {
    // each target has one owner lane per wave: shared-memory H is updated
    // in place, global H by a fire-and-forget reduction
    if (HSM)
      H[h - 1] += x;
    else
      atomicAdd(H + (h - 1), x);
  }
}

// Phase-2 operations and stores, two per lane per step (never aliasing
// within a wave): operands first, then results.
template <typename R, typename Ptr>
__device__ __forceinline__ void eri_coop_load2(const uint4& d, const Ptr& ptr, R (&v)[4]) {
  const int kind = d.x & 3;
  if (kind == 0) {
    v[0] = *ptr(d.y & 0xFFFF);
    v[1] = *ptr(d.y >> 16);
  } else if (kind == 1) {
    const int nt = (d.x >> 2) & 7;
    v[0] = *ptr(d.y & 0xFFFF);
    if (nt > 1) v[1] = *ptr(d.y >> 16);
    if (nt > 2) v[2] = *ptr(d.z & 0xFFFF);
    if (nt > 3) v[3] = *ptr(d.z >> 16);
  } else if (kind == 2) {
    v[0] = *ptr(d.x >> 16);
  }
}

template <bool VOTE, typename R, typename Ptr>
__device__ __forceinline__ void eri_coop_exec2(const uint4& d, const R (&v)[4], const EriPairRec& bra,
                                               const EriPairRec& ket, const EriQuartetRec& qr, double* o, bool acc,
                                               bool red, const double* __restrict__ c2s, const Ptr& ptr) {
  // every lane of the warp calls this; with VOTE the FP64 parts sit behind
  // warp votes (see eri_coop_eval1)
  const int kind = d.x & 3;
  const unsigned dst = d.x >> 16;
  const int nt = kind == 1 ? (d.x >> 2) & 7 : 0;
  if (!VOTE || __any_sync(0xffffffffu, kind == 0)) {
    if (kind == 0) {
      const int ax = d.z;
      const R X = (R)(ax < 3 ? eri_coop_pick3(ax, bra.AB[0], bra.AB[1], bra.AB[2])
                             : eri_coop_pick3(ax - 3, ket.AB[0], ket.AB[1], ket.AB[2]));
      *ptr(dst) = eri_fma(X, v[1], v[0]);
    }
  }
  if (!VOTE || __any_sync(0xffffffffu, nt > 0)) {
    if (nt > 0) {
      R x = (R)__ldg(c2s + (d.w & 255)) * v[0];
      if (nt > 1) x = eri_fma((R)__ldg(c2s + ((d.w >> 8) & 255)), v[1], x);
      if (nt > 2) x = eri_fma((R)__ldg(c2s + ((d.w >> 16) & 255)), v[2], x);
      if (nt > 3) x = eri_fma((R)__ldg(c2s + (d.w >> 24)), v[3], x);
      *ptr(dst) = x;
    }
  }
  if (kind == 2) {
    // the block store (and any accumulation into the output) is FP64
    const int64_t off = (int64_t)(d.z & 255) * qr.st[0] + (int64_t)((d.z >> 8) & 255) * qr.st[1] +
                        (int64_t)((d.z >> 16) & 255) * qr.st[2] + (int64_t)(d.z >> 24) * qr.st[3];
    eri_st(o + off, (double)v[0], acc, red);
  }
}

// Team barrier for a team size known at compile time (TC > 0) or only at
// run time (TC == 0, the persistent launch): __syncwarp for one warp, the
// block barrier for a team that is the whole block (TC >= 128), else the
// named barrier 1 + team with the team's thread count.
template <int TC>
struct EriTeamBarrier {
  int T, tb;
  __device__ __forceinline__ void operator()() const {
    if (TC == 32 || (TC == 0 && T == 32)) {
      __syncwarp();
    } else if (TC >= 128) {
      __syncthreads();  // one team per block
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(1 + tb), "r"(T) : "memory");
    }
  }
};

// One team's quartets: q = q0, q0 + stride, ... < a.nq, each through its
// primitive quartets (Phase 1, wave by wave) and Phase 2 with the stores.
// rows: the team's shared-memory region [coefficient rows | H when hsm |
// value slots]; Hg: the team's private global H otherwise.  TC / HSMC fix
// the team size and the H placement at compile time (HSMC = -1: at run
// time).
// R: value type of the recurrences, the contraction sums H, HRR and the
// transform -- double, or float for the reduced-precision form (coefficient
// rows and the Boys function are still formed in FP64; stores are FP64).
template <typename R, int ILP, bool VOTE, int TC, int HSMC, typename Bar>
__device__ __forceinline__ void eri_coop_team(const EriLaunchArgs& a, const EriCoopArgs& p, const int T_rt,
                                              const bool hsm_rt, const int q0, const int stride, const int l,
                                              R* const rows, R* const Hg, const Bar& team_sync,
                                              const EriFuse* fuse = nullptr, int64_t rec0 = 0,
                                              int* team_word = nullptr) {
  const int T = TC ? TC : T_rt;
  const bool HSM = HSMC >= 0 ? HSMC != 0 : hsm_rt;
  R* const Hsm = rows + p.batch * ERI_COOP_NC;                        // H when HSM
  R* const V = Hsm + (HSM ? p.nh : 0);                              // value slots (shared)
  R* const Hs = HSM ? Hsm : Hg;
  const unsigned nh = (unsigned)p.nh;
  // Phase-2 operand id -> address: H below nh, value slots above
  auto ptr = [&](unsigned id) -> R* { return id < nh ? Hs + id : V + (id - nh); };
  // single: every quartet of the launch has one primitive quartet; a team
  // then computes the coefficient rows of its next p.batch quartets at once
  // (one lane each) rather than one row per quartet on one lane
  const bool single = p.single != 0;
  int gi = 0;  // single: position of quartet q in its group of rows
  for (int q = q0; q < a.nq; q += stride) {
    // Phase 1 needs only the two pairs' primitive ranges; the records' other
    // fields (the A - B displacements, the output offset and strides) are
    // read again for Phase 2, so that they hold no registers through the
    // recurrence
    const int32_t qbra = __ldg(&a.quartets[q].bra), qket = __ldg(&a.quartets[q].ket);
    const int32_t bra_off = __ldg(&a.pairs[ERI_PAIR_INDEX(qbra)].prim_off);
    const int32_t bra_n = __ldg(&a.pairs[ERI_PAIR_INDEX(qbra)].nprim);
    const int32_t ket_off = __ldg(&a.pairs[qket].prim_off);
    const int kk = __ldg(&a.pairs[qket].nprim);
    if (single && gi == 0) {
      const int qi = q + l * stride;
      if (l < p.batch && qi < a.nq) {
        const EriQuartetRec r = a.quartets[qi];
        const auto* const pp = EriPrimsOf<R>::get(a);
        eri_coop_row(pp[a.pairs[ERI_PAIR_INDEX(r.bra)].prim_off], pp[a.pairs[r.ket].prim_off], p.L,
                     a.boys_tab, rows + l * ERI_COOP_NC);
      }
    }
    for (int h = l; h < p.nh; h += T) Hs[h] = (R)0;
    const int k4 = bra_n * kk;
    for (int b0 = 0; b0 < k4; b0 += p.batch) {
      const int nb = min(p.batch, k4 - b0);
      if (!single && l < nb) {
        const int pidx = b0 + l;
        const int i = pidx / kk, j = pidx - (pidx / kk) * kk;
        const auto* const pp = EriPrimsOf<R>::get(a);
        eri_coop_row(pp[bra_off + i], pp[ket_off + j], p.L, a.boys_tab, rows + l * ERI_COOP_NC);
      }
      team_sync();
      for (int pi = 0; pi < nb; ++pi) {
        const R* const row = rows + (single ? gi : pi) * ERI_COOP_NC;
        // a step gives each lane ILP descriptors (independent nodes of the
        // same wave); they are loaded two steps ahead -- the stream ends in
        // two no-op steps -- so the L2 latency overlaps the previous step
        const uint4* dp = p.ph1 + ILP * l;
        uint4 d[ILP], dn[ILP];
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
          d[u] = __ldg(dp + u);
          dn[u] = __ldg(dp + ILP * T + u);
        }
        for (int w = 0; w < p.nw1; ++w) {
          const int steps = (int)__ldg(p.steps1 + w);
          for (int s = 0; s < steps; ++s) {
            uint4 dnn[ILP];
#pragma unroll
            for (int u = 0; u < ILP; ++u) dnn[u] = __ldg(dp + 2 * ILP * T + u);
            dp += ILP * T;
            EriCoopOps<R> v[ILP];
#pragma unroll
            for (int u = 0; u < ILP; ++u) eri_coop_load1(d[u], V, v[u]);
            R x[ILP];
#pragma unroll
            for (int u = 0; u < ILP; ++u) x[u] = eri_coop_eval1<VOTE>(d[u], row, v[u]);
#pragma unroll
            for (int u = 0; u < ILP; ++u) {
              if (HSM)
                eri_coop_store1<true>(d[u], x[u], V, Hsm);
              else
                eri_coop_store1<false>(d[u], x[u], V, Hs);
            }
#pragma unroll
            for (int u = 0; u < ILP; ++u) {
              d[u] = dn[u];
              dn[u] = dnn[u];
            }
          }
          team_sync();
        }
      }
    }
    // Phase 2 and the stores, once per shell quartet
    const EriQuartetRec qr = a.quartets[q];
    const EriPairRec bra = a.pairs[ERI_PAIR_INDEX(qr.bra)];
    const EriPairRec ket = a.pairs[qr.ket];
    const bool acc = ERI_ACCUMULATE(qr.bra);
    const bool red = ERI_REDUCE(qr.bra);
    double* const o = a.out + qr.out_off;
    const uint4* dp = p.ph2 + ILP * l;
    uint4 d[ILP], dn[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      d[u] = __ldg(dp + u);
      dn[u] = __ldg(dp + ILP * T + u);
    }
    for (int w = 0; w < p.nw2; ++w) {
      const int steps = (int)__ldg(p.steps2 + w);
      for (int s = 0; s < steps; ++s) {
        uint4 dnn[ILP];
#pragma unroll
        for (int u = 0; u < ILP; ++u) dnn[u] = __ldg(dp + 2 * ILP * T + u);
        dp += ILP * T;
        R v[ILP][4];
#pragma unroll
        for (int u = 0; u < ILP; ++u) eri_coop_load2(d[u], ptr, v[u]);
#pragma unroll
        for (int u = 0; u < ILP; ++u) eri_coop_exec2<VOTE>(d[u], v[u], bra, ket, qr, o, acc, red, p.c2s, ptr);
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
          d[u] = dn[u];
          dn[u] = dnn[u];
        }
      }
      team_sync();
    }
    if (fuse != nullptr) {
      // J/K of the block once its last part is in: a quartet of several
      // parts (orientations, chunks) is digested by the team that brings its
      // count of finished parts to the total; every lane's stores and
      // reductions reach L2 before the count (fence, then the team barrier
      // that the Phase-2 loop ended with), and the block is read from L2
      const int32_t qu = fuse->rec_q[rec0 + q];
      const int32_t np = fuse->nparts[qu];
      bool last = true;
      if (np > 1) {
        __threadfence();
        team_sync();
        if (l == 0) *team_word = atomicAdd(fuse->done + qu, 1) == np - 1 ? 1 : 0;
        team_sync();
        last = *team_word != 0;
      }
      if (last) {
        __threadfence();
        eri_digest_quartet(fuse->jk, qu, l, T, fuse->jk.blocks + fuse->jk.offsets[qu],
                           [](const double* p) { return __ldcg(p); });
      }
      team_sync();  // team_word is rewritten for the next quartet
    }
    if (single && ++gi == p.batch) gi = 0;
  }
}

// One launch per class bucket.  HSM: the accumulators H share the team's
// shared-memory region with the value slots ([H | slots], operand id =
// offset); otherwise H is a team-private global region and slots follow at
// id - nh.  Blocks are 128 threads (teams of up to 128 lanes) or one team of
// 256 or 512 lanes; every shape keeps the 128 registers per thread that two
// nodes per lane need (four nodes per lane: 255, at most 256 threads per SM).
template <typename R, int T, bool HSM, int ILP, bool VOTE>
__global__ void __launch_bounds__(T > 128 ? T : 128,
                                  T > 256 ? 1 : T > 128 ? (ILP == 4 ? 1 : 2) : (ILP == 4 ? 2 : 4))
    eri_coop_kernel(const EriLaunchArgs a, const EriCoopArgs p) {
  extern __shared__ double eri_coop_smem[];
  const int tb = threadIdx.x / T;           // team within the block
  const int l = threadIdx.x - tb * T;       // lane within the team
  const int team = blockIdx.x * (blockDim.x / T) + tb;
  const int per_team = p.batch * ERI_COOP_NC + (HSM ? p.nh : 0) + p.nslot;
  R* const rows = reinterpret_cast<R*>(eri_coop_smem) + (size_t)tb * per_team;
  R* const Hg = HSM ? nullptr : reinterpret_cast<R*>(p.gH) + (size_t)team * p.nh;
  eri_coop_team<R, ILP, VOTE, T, HSM ? 1 : 0>(a, p, T, HSM, team, p.nteams, l, rows, Hg, EriTeamBarrier<T>{T, tb});
}

// Persistent launch over a device work list (one block of 512 threads per
// SM).  Each item is a run of quartet records of one class program with its
// team shape: the block takes the next item from a global counter, forms
// item.teams teams of item.T lanes (threads beyond them wait for the next
// item), and its teams stride over the item's quartets.  Every cooperative
// class of a plan -- any team size, H placement and vote form -- goes
// through one launch of this kernel per precision.
template <typename R, bool VOTE>
__global__ void __launch_bounds__(512, 1) eri_coop_persist_kernel(const EriLaunchArgs a0, const EriPersistArgs pa) {
  extern __shared__ double eri_coop_smem[];
  // the current item's arguments, read by the teams from shared memory (not
  // held in registers across the item's loops)
  __shared__ EriCoopArgs ps;
  __shared__ EriLaunchArgs as;
  __shared__ EriWorkItem ws;
  __shared__ int item_s;
  __shared__ int team_words[16];  // one per team (fused digestion)
  for (;;) {
    if (threadIdx.x == 0) {
      const int it = atomicAdd(pa.next, 1);
      item_s = it;
      if (it < pa.nitems) {
        const EriWorkItem w = pa.items[it];
        const EriCoopProgDesc g = pa.progs[w.prog];
        ws = w;
        ps.ph1 = g.ph1;
        ps.steps1 = g.steps1;
        ps.ph2 = g.ph2;
        ps.steps2 = g.steps2;
        ps.c2s = pa.c2s;
        ps.gvals = nullptr;
        ps.gH = pa.gH;
        ps.nw1 = g.nw1;
        ps.nw2 = g.nw2;
        ps.nh = g.nh;
        ps.nslot = g.nslot;
        ps.L = g.L;
        ps.smem_slots = g.nslot;
        ps.h_in_smem = w.hsm;
        ps.nteams = w.teams;
        ps.batch = w.batch;
        ps.single = w.single;
        as = a0;
        as.quartets = a0.quartets + w.first;
        as.nq = w.count;
      }
    }
    __syncthreads();
    if (item_s >= pa.nitems) break;
    const int T = ws.T, teams = ws.teams;
    const bool hsm = ws.hsm != 0;
    const int tb = threadIdx.x / T, l = threadIdx.x - tb * T;
    if (tb < teams) {
      const int per_team = ps.batch * ERI_COOP_NC + (hsm ? ps.nh : 0) + ps.nslot;
      R* const rows = reinterpret_cast<R*>(eri_coop_smem) + (size_t)tb * per_team;
      R* const Hg = reinterpret_cast<R*>(pa.gH) + (size_t)blockIdx.x * pa.gh_per_block + (size_t)tb * ps.nh;
      const EriTeamBarrier<0> bar{T, tb};
      eri_coop_team<R, 2, VOTE, 0, -1>(as, ps, T, hsm, tb, teams, l, rows, Hg, bar, pa.fuse.on ? &pa.fuse : nullptr,
                                       (int64_t)ws.first, team_words + tb);
    }
    __syncthreads();  // the item's shared memory is free, the item may be rewritten
  }
}

static const void* const eri_coop_persist_fns[] = {
    (const void*)eri_coop_persist_kernel<double, false>, (const void*)eri_coop_persist_kernel<double, true>,
    (const void*)eri_coop_persist_kernel<float, false>, (const void*)eri_coop_persist_kernel<float, true>};

extern "C" cudaError_t eri_coop_persist_launch(int fp32, int vote, const EriLaunchArgs* a, const EriPersistArgs* pa,
                                               int grid, size_t smem, cudaStream_t stream) {
  EriLaunchArgs aa = *a;
  EriPersistArgs pp = *pa;
  void* args[] = {&aa, &pp};
  return cudaLaunchKernel(eri_coop_persist_fns[2 * (fp32 ? 1 : 0) + (vote ? 1 : 0)], dim3(grid), dim3(512), args,
                          smem, stream);
}

// dynamic shared memory a persistent launch may take: the opt-in limit less
// the static shared memory of its kernels (the current item)
extern "C" size_t eri_coop_persist_smem_max(size_t optin) {
  size_t s = 0;
  for (const void* f : eri_coop_persist_fns) {
    cudaFuncAttributes at;
    if (cudaFuncGetAttributes(&at, f) != cudaSuccess) return 0;
    s = std::max(s, at.sharedSizeBytes);
  }
  return optin - s;
}

#define ERI_COOP_FNS_T(R, I, V)                                                                               \
  (const void*)eri_coop_kernel<R, 32, true, I, V>, (const void*)eri_coop_kernel<R, 32, false, I, V>,           \
      (const void*)eri_coop_kernel<R, 64, true, I, V>, (const void*)eri_coop_kernel<R, 64, false, I, V>,       \
      (const void*)eri_coop_kernel<R, 128, true, I, V>, (const void*)eri_coop_kernel<R, 128, false, I, V>,     \
      (const void*)eri_coop_kernel<R, 256, true, I, V>, (const void*)eri_coop_kernel<R, 256, false, I, V>
// 512-lane teams exist with two nodes per lane only (four would need more
// registers than a 512-thread block can hold)
#define ERI_COOP_FNS_V(R, V)                                                                                   \
  ERI_COOP_FNS_T(R, 2, V), (const void*)eri_coop_kernel<R, 512, true, 2, V>,                                    \
      (const void*)eri_coop_kernel<R, 512, false, 2, V>, ERI_COOP_FNS_T(R, 4, V), nullptr, nullptr

// every instantiation, indexed [vote][fp32][ilp 4][T 32/64/128/256/512][H not in shared memory]
static const void* const eri_coop_fns[] = {ERI_COOP_FNS_V(double, false), ERI_COOP_FNS_V(float, false),
                                           ERI_COOP_FNS_V(double, true), ERI_COOP_FNS_V(float, true)};

extern "C" cudaError_t eri_coop_launch(int T, int ilp, int fp32, int vote, const EriLaunchArgs* a,
                                       const EriCoopArgs* p, int grid, int block, size_t smem, cudaStream_t stream) {
  const int ti = T == 32 ? 0 : T == 64 ? 1 : T == 128 ? 2 : T == 256 ? 3 : T == 512 ? 4 : -1;
  if (ti < 0 || (ilp != 2 && ilp != 4)) return cudaErrorInvalidValue;
  if (block != (T > 128 ? T : 128) && !(T <= 128 && block % T == 0 && block <= 128)) return cudaErrorInvalidValue;
  const int idx = (vote ? 40 : 0) + (fp32 ? 20 : 0) + (ilp == 4 ? 10 : 0) + 2 * ti + (p->h_in_smem ? 0 : 1);
  if (eri_coop_fns[idx] == nullptr) return cudaErrorInvalidValue;
  EriLaunchArgs aa = *a;
  EriCoopArgs pp = *p;
  void* args[] = {&aa, &pp};
  return cudaLaunchKernel(eri_coop_fns[idx], dim3(grid), dim3(block), args, smem, stream);
}

// Diagnostic: F_0..F_L(T[i]) by this tier's Boys routine, one thread per
// argument (F is [n][L + 1]).
__global__ void eri_coop_boys_kernel(const double* __restrict__ T, int64_t n, int L, const double* __restrict__ tab,
                                     double* __restrict__ F) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double f[ERI_BOYS_LMAX + 1];
  eri_coop_boys(L, T[i], f, tab);
  for (int m = 0; m <= L; ++m) F[i * (L + 1) + m] = f[m];
}

extern "C" cudaError_t eri_coop_boys_launch(const double* T, int64_t n, int L, const double* tab, double* F,
                                            cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  eri_coop_boys_kernel<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(T, n, L, tab, F);
  return cudaGetLastError();
}

// shared memory of one coefficient row, in elements, and the largest batch
extern "C" size_t eri_coop_row_elems(void) { return (size_t)ERI_COOP_NC; }
extern "C" int eri_coop_max_batch(void) { return ERI_COOP_BATCH; }

extern "C" cudaError_t eri_coop_set_smem(size_t bytes) {
  for (const void* f : eri_coop_fns) {
    if (f == nullptr) continue;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
  }
  // the persistent kernels hold their current item in static shared memory
  for (const void* f : eri_coop_persist_fns) {
    cudaFuncAttributes at;
    cudaError_t e = cudaFuncGetAttributes(&at, f);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes - at.sharedSizeBytes));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
