// Team-cooperative executor: the tier for large classes (FusionRCG Sec.
// III-C, Regime II, re-derived for GB300).
//
// A team of T lanes (T = 32, 64 or 128; one to four warps) evaluates one
// shell quartet: it walks the quartet's primitive quartets one at a time
// (Algorithm 2's loops, accumulate-then-transform), and for each it runs the
// Phase-1 graph wave by wave -- every wave is a set of up to T mutually
// independent nodes in DSA order (Eq. 7), lane l takes node l -- with a team
// barrier between waves.  Phase 2 (HRR + stepwise transform, Eq. 16) and the
// output stores run the same way once per shell quartet.
//
// The value slots of one primitive quartet are shared by the whole team, so
// a class whose live set is thousands of values stays in shared memory; the
// accumulator bank H sits in shared memory when it fits, else in a
// team-private global region (L2-resident).  Operand ids: id < nh is H[id],
// id >= nh is value slot id - nh; slots beyond the shared-memory part spill to
// a team-private global region.
#include "eri_common.cuh"

struct EriCoopArgs {
  const uint4* __restrict__ ph1;      // Phase-1 descriptors, waves of steps x T
  const uint32_t* __restrict__ steps1;
  const uint4* __restrict__ ph2;      // Phase-2 descriptors
  const uint32_t* __restrict__ steps2;
  const double* __restrict__ c2s;     // transform coefficient table
  double* __restrict__ gvals;         // [team][nslot - smem_slots] value slots beyond shared memory
  double* __restrict__ gH;            // [team][nh] when H is not in shared memory
  int32_t nw1, nw2;
  int32_t nh, nslot, L;
  int32_t smem_slots;                 // value slots held in shared memory
  int32_t h_in_smem;
  int32_t nteams;                     // teams in the grid
};

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

template <int T>
__device__ __forceinline__ void eri_team_sync() {
  if (T == 32) {
    __syncwarp();
  } else if (T == 128) {
    __syncthreads();
  } else {
    // two teams of 64 lanes per 128-thread block: named barriers 1 and 2
    asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(threadIdx.x / T)), "r"(T) : "memory");
  }
}

template <int T>
__global__ void __launch_bounds__(128) eri_coop_kernel(const EriLaunchArgs a, const EriCoopArgs p) {
  extern __shared__ double eri_coop_smem[];
  const int tb = threadIdx.x / T;           // team within the block
  const int l = threadIdx.x - tb * T;       // lane within the team
  const int team = blockIdx.x * (128 / T) + tb;
  const int per_team = p.smem_slots + (p.h_in_smem ? p.nh : 0);
  double* const Vs = eri_coop_smem + (size_t)tb * per_team;
  double* const Hs = p.h_in_smem ? Vs + p.smem_slots : p.gH + (size_t)team * p.nh;
  double* const Vg = p.gvals + (size_t)team * (p.nslot - p.smem_slots);
  const unsigned nh = (unsigned)p.nh, ns = (unsigned)p.smem_slots;
  // operand id -> address (per lane; ids differ between lanes)
  auto ptr = [&](unsigned id) -> double* {
    if (id < nh) return Hs + id;
    id -= nh;
    return id < ns ? Vs + id : Vg + (id - ns);
  };
  for (int q = team; q < a.nq; q += p.nteams) {
    const EriQuartetRec qr = a.quartets[q];
    const EriPairRec bra = a.pairs[ERI_PAIR_INDEX(qr.bra)];
    const bool acc = ERI_ACCUMULATE(qr.bra);
    const EriPairRec ket = a.pairs[qr.ket];
    for (int h = l; h < p.nh; h += T) Hs[h] = 0.0;
    eri_team_sync<T>();
    const int kk = ket.nprim;
    for (int i = 0, j = 0; i < bra.nprim;) {
      const EriPairPrim bp = a.pprims[bra.prim_off + i];
      const EriPairPrim kp = a.pprims[ket.prim_off + j];
      if (++j == kk) {
        j = 0;
        ++i;
      }
      EriPrimQuartet pq;
      eri_prim_quartet(bp, kp, pq);
      double F[ERI_BOYS_LMAX + 1];
      eri_coop_boys(p.L, pq.T, F, a.boys_tab);
      double c1b[8], c1k[8], c3[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        c1b[k] = (double)(k + 1) * bp.inv2z;
        c1k[k] = (double)(k + 1) * kp.inv2z;
        c3[k] = (double)(k + 1) * (0.5 * pq.s);
      }
      const double roz = -pq.te, roe = -pq.tz;
      const uint4* d1 = p.ph1 + l;
      for (int w = 0; w < p.nw1; ++w) {
        const int steps = (int)__ldg(p.steps1 + w);
        for (int s = 0; s < steps; ++s, d1 += T) {
          const uint4 d = __ldg(d1);
          const int side = (d.w >> 16) & 3;
          if (side == 3) continue;
          const int k = (d.w >> 20) & 31;
          double x;
          if (side == 2) {
            x = pq.pref * F[k];
          } else {
            const int axis = (d.w >> 18) & 3;
            const int k3 = (d.w >> 25) & 31;
            const double cg = side ? eri_coop_pick3(axis, kp.PA[0], kp.PA[1], kp.PA[2])
                                   : eri_coop_pick3(axis, bp.PA[0], bp.PA[1], bp.PA[2]);
            const double cw = side ? eri_coop_pick3(axis, pq.WQ[0], pq.WQ[1], pq.WQ[2])
                                   : eri_coop_pick3(axis, pq.WP[0], pq.WP[1], pq.WP[2]);
            x = cg * *ptr(d.y & 0xFFFF);
            x = fma(cw, *ptr(d.y >> 16), x);
            if (k) {
              const double ck = side ? eri_coop_pick8(k, c1k) : eri_coop_pick8(k, c1b);
              const double t = fma(side ? roe : roz, *ptr(d.z >> 16), *ptr(d.z & 0xFFFF));
              x = fma(ck, t, x);
            }
            if (k3) x = fma(eri_coop_pick8(k3, c3), *ptr(d.w & 0xFFFF), x);
          }
          if (d.w & (1u << 30)) *ptr(d.x & 0xFFFF) = x;
          const unsigned h = d.x >> 16;
          if (h) Hs[h - 1] += x;
        }
        eri_team_sync<T>();
      }
    }
    // Phase 2 and the stores, once per shell quartet
    double* const o = a.out + qr.out_off;
    const uint4* d2 = p.ph2 + l;
    for (int w = 0; w < p.nw2; ++w) {
      const int steps = (int)__ldg(p.steps2 + w);
      for (int s = 0; s < steps; ++s, d2 += T) {
        const uint4 d = __ldg(d2);
        const int kind = d.x & 3;
        if (kind == 3) continue;
        const unsigned dst = d.x >> 16;
        if (kind == 0) {
          const int ax = d.z;
          const double X = ax < 3 ? eri_coop_pick3(ax, bra.AB[0], bra.AB[1], bra.AB[2])
                                  : eri_coop_pick3(ax - 3, ket.AB[0], ket.AB[1], ket.AB[2]);
          *ptr(dst) = fma(X, *ptr(d.y >> 16), *ptr(d.y & 0xFFFF));
        } else if (kind == 1) {
          const int nt = (d.x >> 2) & 7;
          double x = __ldg(p.c2s + (d.w & 255)) * *ptr(d.y & 0xFFFF);
          if (nt > 1) x = fma(__ldg(p.c2s + ((d.w >> 8) & 255)), *ptr(d.y >> 16), x);
          if (nt > 2) x = fma(__ldg(p.c2s + ((d.w >> 16) & 255)), *ptr(d.z & 0xFFFF), x);
          if (nt > 3) x = fma(__ldg(p.c2s + (d.w >> 24)), *ptr(d.z >> 16), x);
          *ptr(dst) = x;
        } else {
          const int64_t off = (int64_t)(d.z & 255) * qr.st[0] + (int64_t)((d.z >> 8) & 255) * qr.st[1] +
                              (int64_t)((d.z >> 16) & 255) * qr.st[2] + (int64_t)(d.z >> 24) * qr.st[3];
          eri_st(o + off, *ptr(dst), acc);
        }
      }
      eri_team_sync<T>();
    }
  }
}

extern "C" cudaError_t eri_coop_launch(int T, const EriLaunchArgs* a, const EriCoopArgs* p, int grid, size_t smem,
                                       cudaStream_t stream) {
  switch (T) {
    case 32:
      eri_coop_kernel<32><<<grid, 128, smem, stream>>>(*a, *p);
      break;
    case 64:
      eri_coop_kernel<64><<<grid, 128, smem, stream>>>(*a, *p);
      break;
    case 128:
      eri_coop_kernel<128><<<grid, 128, smem, stream>>>(*a, *p);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

extern "C" cudaError_t eri_coop_set_smem(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(eri_coop_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(eri_coop_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(eri_coop_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return e;
}
