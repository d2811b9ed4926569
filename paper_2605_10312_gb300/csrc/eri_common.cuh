// Device-side data layout and helpers shared by the runtime and the
// generated class kernels of the contracted-ERI path.
//
// Everything a class kernel reads is prepared on the device by the pair
// set-up kernel (FusionRCG Algorithm 2, "GaussianPairs", hoisted out of the
// primitive loop to once per primitive pair):
//   EriPairPrim  per primitive pair (a_i, b_j) of an oriented shell pair
//   EriPairRec   per oriented shell pair: its primitive pairs and A - B
//   EriQuartetRec per shell quartet: its bra and ket pairs and where and
//                how its block is written
#pragma once
#include <stdint.h>

struct EriPairPrim {   // 72 bytes
  double zeta;         // a_i + b_j
  double inv2z;        // 1 / (2 zeta)
  double P[3];         // (a_i A + b_j B) / zeta
  double PA[3];        // P - A  (A = the recurrence centre of the pair)
  double K;            // sqrt(2) pi^(5/4) c_i N_i c_j N_j exp(-a_i b_j |A-B|^2 / zeta) / zeta
};

// The same quantities rounded to FP32, for quartets whose recurrences run
// in FP32 (written by the pair set-up kernel beside the FP64 record).  P is
// kept as an unevaluated sum P_hi + P_lo of two floats, so that P - Q of
// two pairs keeps FP32 relative accuracy when P and Q are close (a plain
// float P would lose it to cancellation at coordinates of tens of bohr).
struct EriPairPrimF {  // 48 bytes
  float zeta;
  float inv2z;
  float Phi[3], Plo[3];
  float PA[3];
  float K;
};

__device__ __forceinline__ EriPairPrimF eri_pair_prim_f32(const EriPairPrim& q) {
  EriPairPrimF f;
  f.zeta = (float)q.zeta;
  f.inv2z = (float)q.inv2z;
  for (int d = 0; d < 3; ++d) {
    f.Phi[d] = (float)q.P[d];
    f.Plo[d] = (float)(q.P[d] - (double)f.Phi[d]);
    f.PA[d] = (float)q.PA[d];
  }
  f.K = (float)q.K;
  return f;
}

struct EriPairRec {    // 32 bytes
  int32_t prim_off;    // first EriPairPrim
  int32_t nprim;       // K_a * K_b
  double AB[3];        // A - B
};

struct EriQuartetRec { // 32 bytes
  int32_t bra, ket;    // EriPairRec indices (bra = centres A, B; ket = C, D);
                       // bit 31 of bra: add into the block instead of writing it
  int64_t out_off;     // first output element of this quartet's block
  int32_t st[4];       // output strides of the A, B, C, D component indices
};

#define ERI_PAIR_INDEX(x) ((x) & 0x3fffffff)
#define ERI_ACCUMULATE(x) ((x) < 0)
#define ERI_REDUCE(x) (((x) >> 30) & 1)

// Output store of one element.  The first part of a quartet writes its
// block, later parts (other pair orientations, later launches) add to it;
// chunks of one quartet that run concurrently in one launch reduce into a
// block the launch zeroed first.
__device__ __forceinline__ void eri_st(double* p, double v, bool acc) { *p = acc ? *p + v : v; }
__device__ __forceinline__ void eri_st(double* p, double v, bool acc, bool red) {
  if (red)
    atomicAdd(p, v);
  else
    *p = acc ? *p + v : v;
}

struct EriLaunchArgs {
  const EriQuartetRec* __restrict__ quartets;  // this launch's quartets
  const EriPairRec* __restrict__ pairs;
  const EriPairPrim* __restrict__ pprims;
  const EriPairPrimF* __restrict__ pprims_f;   // FP32 copy (plans with FP32 quartets, else null)
  const double* __restrict__ boys_tab;         // Taylor table, see below
  double* __restrict__ out;
  double* __restrict__ scratch;                // slot tiers: [slot][thread]
  int64_t scratch_stride;                      // doubles between slots
  int32_t nq;
  int32_t group;                               // lanes sharing one shell quartet (1, 2, 4, .. 32)
};

// Lanes [base, base + group) of a warp cooperate on one shell quartet; this
// is their member mask for the warp-synchronous primitives.
__device__ __forceinline__ unsigned eri_group_mask(int group) {
  if (group >= 32) return 0xffffffffu;
  const int lane = threadIdx.x & 31;
  return ((1u << group) - 1u) << (lane & ~(group - 1));
}

// Program-driven tiers: one class program (descriptor streams, see the
// generator's encode module) and the transform coefficient table.
struct EriProgArgs {
  const uint4* __restrict__ ph1;   // Phase-1 descriptors
  const uint4* __restrict__ ph2;   // Phase-2 descriptors
  const double* __restrict__ c2s;  // transform coefficient table
  int32_t n1, n2;
  int32_t nh;                      // accumulators, slots [0, nh)
  int32_t L;                       // la + lb + lc + ld
};

// ---------------------------------------------------------------------------
// Boys function F_m(T), m = 0..L   (base values of Phase 1, Sec. II-A)
//
// T < ERI_BOYS_TMAX: Taylor expansion about the nearest grid point T_k = k h,
//   F_L(T_k + d) = sum_{j<ERI_BOYS_NTAY} F_{L+j}(T_k) (-d)^j / j!,  |d| <= h/2,
//   then downward recursion F_m = (2T F_{m+1} + exp(-T)) / (2m+1)
//   (the interpolation scheme of Gill, Johnson and Pople, Int. J. Quantum
//   Chem. 40, 745 (1991); table values from high-precision quadrature).
// T >= ERI_BOYS_TMAX: F_0 = sqrt(pi/T)/2 (erf(sqrt T) = 1 to double
//   precision there) and upward recursion F_{m+1} = ((2m+1) F_m - exp(-T))/(2T),
//   which is stable for T > m.
// ---------------------------------------------------------------------------
#define ERI_BOYS_STEP 0.1
#define ERI_BOYS_INV_STEP 10.0
#define ERI_BOYS_TMAX 36.0
#define ERI_BOYS_NGRID 362          // k = 0..361
#define ERI_BOYS_NTAY 8             // Taylor terms
#define ERI_BOYS_LMAX 16            // highest order the kernels need
#define ERI_BOYS_NCOL (ERI_BOYS_LMAX + ERI_BOYS_NTAY)   // orders 0..23 per grid point

// 1 / (2m + 1), m = 0..ERI_BOYS_LMAX (a per-translation-unit constant table)
static __constant__ double eri_inv_odd[ERI_BOYS_LMAX + 1] = {
    1.0, 1.0 / 3, 1.0 / 5, 1.0 / 7, 1.0 / 9, 1.0 / 11, 1.0 / 13, 1.0 / 15, 1.0 / 17,
    1.0 / 19, 1.0 / 21, 1.0 / 23, 1.0 / 25, 1.0 / 27, 1.0 / 29, 1.0 / 31, 1.0 / 33};

template <int L>
__device__ __forceinline__ void eri_boys(double T, double (&F)[L + 1], const double* __restrict__ tab) {
  const double ex = exp(-T);
  if (T < ERI_BOYS_TMAX) {
    const int k = __double2int_rn(T * ERI_BOYS_INV_STEP);
    const double d = T - k * ERI_BOYS_STEP;
    const double* r = tab + k * ERI_BOYS_NCOL + L;
    // Horner in (-d): c_j = F_{L+j}(T_k) / j!
    double acc = __ldg(r + ERI_BOYS_NTAY - 1);
#pragma unroll
    for (int j = ERI_BOYS_NTAY - 1; j >= 1; --j) acc = fma(acc, -d * (1.0 / j), __ldg(r + j - 1));
    F[L] = acc;
#pragma unroll
    for (int m = L - 1; m >= 0; --m) F[m] = fma(2.0 * T, F[m + 1], ex) * (1.0 / (2 * m + 1));
  } else {
    const double rt = rsqrt(T);
    F[0] = 0.88622692545275801365 * rt;  // sqrt(pi)/2 / sqrt(T)
    const double h = 0.5 * rt * rt;      // 1 / (2T)
#pragma unroll
    for (int m = 0; m < L; ++m) F[m + 1] = fma((double)(2 * m + 1), F[m], -ex) * h;
  }
}

// Per-primitive-quartet quantities shared by every class kernel.
struct EriPrimQuartet {
  double s;        // 1 / (zeta + eta)
  double te, tz;   // eta s = rho/zeta,  zeta s = rho/eta
  double WP[3];    // W - P
  double WQ[3];    // W - Q
  double T;        // rho |P - Q|^2
  double pref;     // K_ab K_cd / sqrt(zeta + eta)
};

__device__ __forceinline__ void eri_prim_quartet(const EriPairPrim& b, const EriPairPrim& k, EriPrimQuartet& o) {
  const double s = 1.0 / (b.zeta + k.zeta);
  const double te = k.zeta * s, tz = b.zeta * s;
  const double pq0 = b.P[0] - k.P[0], pq1 = b.P[1] - k.P[1], pq2 = b.P[2] - k.P[2];
  o.s = s;
  o.te = te;
  o.tz = tz;
  o.WP[0] = -te * pq0; o.WP[1] = -te * pq1; o.WP[2] = -te * pq2;
  o.WQ[0] = tz * pq0;  o.WQ[1] = tz * pq1;  o.WQ[2] = tz * pq2;
  const double rho = b.zeta * te;
  o.T = rho * fma(pq0, pq0, fma(pq1, pq1, pq2 * pq2));
  o.pref = b.K * k.K * sqrt(s);
}

// The same in FP32, for quartets whose recurrences run in FP32: only the
// Boys function (and the accumulation into the block) stays in FP64.
struct EriPrimQuartetF {
  float s, te, tz;
  float WP[3], WQ[3];
  float T, pref;
};

__device__ __forceinline__ void eri_prim_quartet_f32(const EriPairPrimF& b, const EriPairPrimF& k,
                                                     EriPrimQuartetF& o) {
  const float s = 1.0f / (b.zeta + k.zeta);
  const float te = k.zeta * s, tz = b.zeta * s;
  float pq[3];
  for (int d = 0; d < 3; ++d) pq[d] = (b.Phi[d] - k.Phi[d]) + (b.Plo[d] - k.Plo[d]);
  o.s = s;
  o.te = te;
  o.tz = tz;
  for (int d = 0; d < 3; ++d) {
    o.WP[d] = -te * pq[d];
    o.WQ[d] = tz * pq[d];
  }
  const float rho = b.zeta * te;
  o.T = rho * fmaf(pq[0], pq[0], fmaf(pq[1], pq[1], pq[2] * pq[2]));
  o.pref = b.K * k.K * sqrtf(s);
}
