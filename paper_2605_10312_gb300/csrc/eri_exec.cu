// Program-driven executor: one compiled kernel that runs the straight-line
// class program the generator encoded (FusionRCG Sec. III-A schedule,
// Sec. III-B stepwise transform, Sec. III-C tiering).
//
// One thread evaluates one shell quartet (Algorithm 2).  Every lane of a warp
// walks the same descriptor stream, so each descriptor is a broadcast load;
// decoding and slot addressing run on the integer pipes while the FP64 pipe,
// the bound of this kernel on GB300, does only the recurrence arithmetic.
//
// Value slots live either in shared memory ([slot][thread], the shared
// tier) or in a global scratch interleaved across the grid ([slot][thread],
// the global tier; the paper's coalesced Tier-2 buffer).  The kernel is
// persistent: the grid is sized to the machine and threads stride over the
// quartets of their launch.
#include "eri_common.cuh"

// k-th entry (k = 1..8) of a uniform 8-entry register table; k is the same in
// every lane, so this is a short select chain on the integer pipes.
__device__ __forceinline__ double eri_pick8(int k, const double (&t)[8]) {
  double r = t[0];
#pragma unroll
  for (int i = 1; i < 8; ++i) r = (k == i + 1) ? t[i] : r;
  return r;
}

__device__ __forceinline__ double eri_pick3(int i, double x, double y, double z) {
  return i == 0 ? x : (i == 1 ? y : z);
}

// Boys values for a run-time order L (the executor serves every class).
__device__ __forceinline__ void eri_boys_rt(int L, double T, double* F, const double* __restrict__ tab) {
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

template <int SHARED>
__global__ void __launch_bounds__(128) eri_exec_kernel(const EriLaunchArgs a, const EriProgArgs p) {
  extern __shared__ double eri_exec_smem[];
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  // a.group lanes of a warp share one shell quartet: each takes every
  // G-th primitive quartet into its own accumulators, the group then sums
  // them and lane 0 runs Phase 2
  const int G = a.group;
  const int r = gt & (G - 1);
  const int ngroups = (gridDim.x * blockDim.x) / G;
  const unsigned gmask = eri_group_mask(G);
  double* const V = SHARED ? eri_exec_smem + threadIdx.x : a.scratch + gt;
  const int64_t vs = SHARED ? (int64_t)blockDim.x : a.scratch_stride;
#define VAL(s) V[(int64_t)(s) * vs]
  for (int q = gt / G; q < a.nq; q += ngroups) {
    const EriQuartetRec qr = a.quartets[q];
    const EriPairRec bra = a.pairs[ERI_PAIR_INDEX(qr.bra)];
    const bool acc = ERI_ACCUMULATE(qr.bra);
    const bool red = ERI_REDUCE(qr.bra);
    const EriPairRec ket = a.pairs[qr.ket];
    for (int h = 0; h < p.nh; ++h) VAL(h) = 0.0;
    const int kk = ket.nprim;
    int i = r / kk, j = r - (r / kk) * kk;
    while (i < bra.nprim) {
      const EriPairPrim bp = a.pprims[bra.prim_off + i];
      const EriPairPrim kp = a.pprims[ket.prim_off + j];
      j += G;
      while (j >= kk) {
        j -= kk;
        ++i;
      }
      EriPrimQuartet pq;
      eri_prim_quartet(bp, kp, pq);
      double F[ERI_BOYS_LMAX + 1];
      eri_boys_rt(p.L, pq.T, F, a.boys_tab);
      // k/(2 zeta), k/(2 eta), k/(2 (zeta + eta)) for k = 1..8, and the
      // factors -rho/zeta, -rho/eta of the second Obara-Saika term
      double c1b[8], c1k[8], c3[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        c1b[k] = (double)(k + 1) * bp.inv2z;
        c1k[k] = (double)(k + 1) * kp.inv2z;
        c3[k] = (double)(k + 1) * (0.5 * pq.s);
      }
      const double roz = -pq.te, roe = -pq.tz;
      for (int n = 0; n < p.n1; ++n) {
        const uint4 d = __ldg(p.ph1 + n);
        const int side = (d.w >> 16) & 3;
        const int k = (d.w >> 20) & 31;
        double x;
        if (side == 2) {
          x = pq.pref * F[k];
        } else {
          const int axis = (d.w >> 18) & 3;
          const int k3 = (d.w >> 25) & 31;
          const double cg = side ? eri_pick3(axis, kp.PA[0], kp.PA[1], kp.PA[2])
                                 : eri_pick3(axis, bp.PA[0], bp.PA[1], bp.PA[2]);
          const double cw = side ? eri_pick3(axis, pq.WQ[0], pq.WQ[1], pq.WQ[2])
                                 : eri_pick3(axis, pq.WP[0], pq.WP[1], pq.WP[2]);
          x = cg * VAL(d.y & 0xFFFF);
          x = fma(cw, VAL(d.y >> 16), x);
          if (k) {
            const double ck = side ? eri_pick8(k, c1k) : eri_pick8(k, c1b);
            const double t = fma(side ? roe : roz, VAL(d.z >> 16), VAL(d.z & 0xFFFF));
            x = fma(ck, t, x);
          }
          if (k3) x = fma(eri_pick8(k3, c3), VAL(d.w & 0xFFFF), x);
        }
        if (d.w & (1u << 30)) VAL(d.x & 0xFFFF) = x;
        const unsigned h = d.x >> 16;
        if (h) VAL(h - 1) += x;
      }
    }
    if (G > 1) {
      // sum the group's accumulators into lane 0's: lane r takes h = r mod G
      __syncwarp(gmask);
      double* const V0 = V - r;  // lanes of a group are adjacent columns
      for (int h = r; h < p.nh; h += G) {
        double s = V0[(int64_t)h * vs];
        for (int l = 1; l < G; ++l) s += V0[(int64_t)h * vs + l];
        V0[(int64_t)h * vs] = s;
      }
      __syncwarp(gmask);
    }
    if (r == 0) {
      // Phase 2: HRR and the stepwise transform, then the stores
      double* const o = a.out + qr.out_off;
      for (int n = 0; n < p.n2; ++n) {
        const uint4 d = __ldg(p.ph2 + n);
        const int kind = d.x & 3;
        const unsigned dst = d.x >> 16;
        if (kind == 0) {
          const int ax = d.z;
          const double X = ax < 3 ? eri_pick3(ax, bra.AB[0], bra.AB[1], bra.AB[2])
                                  : eri_pick3(ax - 3, ket.AB[0], ket.AB[1], ket.AB[2]);
          VAL(dst) = fma(X, VAL(d.y >> 16), VAL(d.y & 0xFFFF));
        } else if (kind == 1) {
          const int nt = (d.x >> 2) & 7;
          double x = ((d.x >> 5) & 1) ? VAL(dst) : 0.0;
          x = fma(__ldg(p.c2s + (d.w & 255)), VAL(d.y & 0xFFFF), x);
          if (nt > 1) x = fma(__ldg(p.c2s + ((d.w >> 8) & 255)), VAL(d.y >> 16), x);
          if (nt > 2) x = fma(__ldg(p.c2s + ((d.w >> 16) & 255)), VAL(d.z & 0xFFFF), x);
          if (nt > 3) x = fma(__ldg(p.c2s + (d.w >> 24)), VAL(d.z >> 16), x);
          VAL(dst) = x;
        } else {
          const int64_t off = (int64_t)(d.z & 255) * qr.st[0] + (int64_t)((d.z >> 8) & 255) * qr.st[1] +
                              (int64_t)((d.z >> 16) & 255) * qr.st[2] + (int64_t)(d.z >> 24) * qr.st[3];
          eri_st(o + off, VAL(dst), acc, red);
        }
      }
    }
    // the group's lanes do not touch lane 0's slots again before the next
    // reduction, which comes after a warp-synchronous point
    if (G > 1) __syncwarp(gmask);
  }
#undef VAL
}

// Diagnostic: F_0..F_L(T[i]) by this tier's Boys routine, one thread per
// argument (F is [n][L + 1]).
__global__ void eri_exec_boys_kernel(const double* __restrict__ T, int64_t n, int L, const double* __restrict__ tab,
                                     double* __restrict__ F) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double f[ERI_BOYS_LMAX + 1];
  eri_boys_rt(L, T[i], f, tab);
  for (int m = 0; m <= L; ++m) F[i * (L + 1) + m] = f[m];
}

extern "C" cudaError_t eri_exec_boys_launch(const double* T, int64_t n, int L, const double* tab, double* F,
                                            cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  eri_exec_boys_kernel<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(T, n, L, tab, F);
  return cudaGetLastError();
}

extern "C" cudaError_t eri_exec_launch(int shared, const EriLaunchArgs* a, const EriProgArgs* p, int grid,
                                       int block, size_t smem, cudaStream_t stream) {
  if (shared) {
    eri_exec_kernel<1><<<grid, block, smem, stream>>>(*a, *p);
  } else {
    eri_exec_kernel<0><<<grid, block, 0, stream>>>(*a, *p);
  }
  return cudaGetLastError();
}

extern "C" cudaError_t eri_exec_set_smem(size_t bytes) {
  return cudaFuncSetAttribute(eri_exec_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
