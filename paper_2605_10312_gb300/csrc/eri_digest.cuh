// Coulomb and exchange digestion of one contracted ERI block (the six
// small contractions described in eri_digest.cu), shared by the separate
// digestion kernels and the fused epilogue of the persistent cooperative
// launch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct EriDigestArgs {
  const int64_t* __restrict__ list;      // quartets this launch digests (indices into quartets)
  int64_t nlist;
  const int32_t* __restrict__ quartets;  // [nq][4] shell indices, the caller's order
  const int64_t* __restrict__ offsets;   // [nq + 1] first element of each block, and the total
  const int32_t* __restrict__ shell_bf;  // [nshell + 1] first basis function of each shell
  const double* __restrict__ blocks;
  const double* __restrict__ D;          // [nbf][nbf], symmetric
  double* J;                             // [nbf][nbf] or null
  double* K;                             // [nbf][nbf] or null
  int64_t nq;
  int32_t nbf;
  int32_t tri;  // 1: J and K are triangle scratch (one reduction per mirrored pair, see eri_jk_add)
};

// Add s to M_rc and M_cr (every J and K contribution comes in such mirrored
// pairs).  tri: only the entry with r <= c receives the pair (2 s on the
// diagonal), halving the reductions; the triangle is folded into the
// caller's full matrix afterwards.
__device__ __forceinline__ void eri_jk_add(double* M, int64_t n, int64_t r, int64_t c, double s, bool tri) {
  if (tri) {
    if (r > c) {
      const int64_t t = r;
      r = c;
      c = t;
    }
    atomicAdd(M + r * n + c, r == c ? 2.0 * s : s);
  } else {
    atomicAdd(M + r * n + c, s);
    atomicAdd(M + c * n + r, s);
  }
}

// number of the 8 index permutations that map (a b | c d) onto itself
__device__ __forceinline__ int eri_stabilizer(int a, int b, int c, int d) {
  int n = 1;                                   // (ab|cd)
  n += (a == b);                               // (ba|cd)
  n += (c == d);                               // (ab|dc)
  n += (a == b && c == d);                     // (ba|dc)
  n += (a == c && b == d);                     // (cd|ab)
  n += (a == d && b == c);                     // (dc|ba)
  n += (a == b && b == c && c == d);           // (dc|ab): d = a, c = b, a = c, b = d
  n += (a == b && b == c && c == d);           // (cd|ba): c = a, d = b, b = c, a = d
  return n;
}

// Digest quartet q from its block v; the W threads lane = 0..W-1 of a group
// share its output entries (W = 1: one thread does all of them).  LD loads a
// block element (plain, or bypassing L1 for blocks other SMs reduced into).
template <typename LD>
__device__ __forceinline__ void eri_digest_quartet(const EriDigestArgs& g, int64_t q, int lane, int W,
                                                   const double* __restrict__ v, LD ld) {
  const int a = g.quartets[4 * q], b = g.quartets[4 * q + 1], c = g.quartets[4 * q + 2], d = g.quartets[4 * q + 3];
  const int A = g.shell_bf[a], B = g.shell_bf[b], C = g.shell_bf[c], Dd = g.shell_bf[d];
  const int na = g.shell_bf[a + 1] - A, nb = g.shell_bf[b + 1] - B, nc = g.shell_bf[c + 1] - C,
            nd = g.shell_bf[d + 1] - Dd;
  const double f = 1.0 / (double)eri_stabilizer(a, b, c, d);
  const double* __restrict__ Dm = g.D;
  const bool tri = g.tri != 0;
  const int64_t n = g.nbf;
  const int sj = nc * nd, si = nb * sj;  // strides of i and j in the block; k stride nd
  if (g.J) {
    // Jab[i][j] = 2 f sum_kl v D_kl
    for (int o = lane; o < na * nb; o += W) {
      const int i = o / nb, j = o - i * nb;
      const double* r = v + (int64_t)i * si + (int64_t)j * sj;
      double s = 0.0;
      for (int k = 0; k < nc; ++k)
        for (int l = 0; l < nd; ++l) s = fma(ld(r + k * nd + l), __ldg(Dm + (C + k) * n + Dd + l), s);
      s *= 2.0 * f;
      eri_jk_add(g.J, n, A + i, B + j, s, tri);
    }
    // Jcd[k][l] = 2 f sum_ij v D_ij
    for (int o = lane; o < nc * nd; o += W) {
      const int k = o / nd, l = o - k * nd;
      double s = 0.0;
      for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j)
          s = fma(ld(v + (int64_t)i * si + (int64_t)j * sj + o), __ldg(Dm + (A + i) * n + B + j), s);
      s *= 2.0 * f;
      eri_jk_add(g.J, n, C + k, Dd + l, s, tri);
    }
  }
  if (g.K) {
    // Kac[i][k] = f sum_jl v D_jl
    for (int o = lane; o < na * nc; o += W) {
      const int i = o / nc, k = o - i * nc;
      double s = 0.0;
      for (int j = 0; j < nb; ++j)
        for (int l = 0; l < nd; ++l)
          s = fma(ld(v + (int64_t)i * si + (int64_t)j * sj + k * nd + l), __ldg(Dm + (B + j) * n + Dd + l), s);
      s *= f;
      eri_jk_add(g.K, n, A + i, C + k, s, tri);
    }
    // Kad[i][l] = f sum_jk v D_jk
    for (int o = lane; o < na * nd; o += W) {
      const int i = o / nd, l = o - i * nd;
      double s = 0.0;
      for (int j = 0; j < nb; ++j)
        for (int k = 0; k < nc; ++k)
          s = fma(ld(v + (int64_t)i * si + (int64_t)j * sj + k * nd + l), __ldg(Dm + (B + j) * n + C + k), s);
      s *= f;
      eri_jk_add(g.K, n, A + i, Dd + l, s, tri);
    }
    // Kbc[j][k] = f sum_il v D_il
    for (int o = lane; o < nb * nc; o += W) {
      const int j = o / nc, k = o - j * nc;
      double s = 0.0;
      for (int i = 0; i < na; ++i)
        for (int l = 0; l < nd; ++l)
          s = fma(ld(v + (int64_t)i * si + (int64_t)j * sj + k * nd + l), __ldg(Dm + (A + i) * n + Dd + l), s);
      s *= f;
      eri_jk_add(g.K, n, B + j, C + k, s, tri);
    }
    // Kbd[j][l] = f sum_ik v D_ik
    for (int o = lane; o < nb * nd; o += W) {
      const int j = o / nd, l = o - j * nd;
      double s = 0.0;
      for (int i = 0; i < na; ++i)
        for (int k = 0; k < nc; ++k)
          s = fma(ld(v + (int64_t)i * si + (int64_t)j * sj + k * nd + l), __ldg(Dm + (A + i) * n + C + k), s);
      s *= f;
      eri_jk_add(g.K, n, B + j, Dd + l, s, tri);
    }
  }
}

