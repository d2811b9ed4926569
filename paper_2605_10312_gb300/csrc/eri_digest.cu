// Coulomb and exchange digestion of contracted ERI blocks (FusionRCG
// Alg. 2, the scatter of each quartet's integrals into the Fock build):
//
//   J_ij += sum_kl (ij|kl) D_kl,      K_ij += sum_kl (ik|jl) D_kl
//
// for a symmetric density D, from blocks of shell quartets that each stand
// for their orbit under the 8 index permutations (ab|cd) = (ba|cd) =
// (ab|dc) = (cd|ab) = ...  A quartet whose shells coincide under some of
// those permutations (a = b, c = d, (ab) = (cd), ...) is weighted by the
// inverse of the number of permutations that leave it unchanged, so that
// every ordered element of the full tensor is counted once.
//
// Summing the 8 permutations of one element (ij|kl) with D symmetric gives
// six small contractions per quartet block v[i][j][k][l]:
//   Jab[i][j] = 2 f sum_kl v D_kl   -> J_ij and J_ji
//   Jcd[k][l] = 2 f sum_ij v D_ij   -> J_kl and J_lk
//   Kac[i][k] =   f sum_jl v D_jl   -> K_ik and K_ki
//   Kad[i][l] =   f sum_jk v D_jk   -> K_il and K_li
//   Kbc[j][k] =   f sum_il v D_il   -> K_jk and K_kj
//   Kbd[j][l] =   f sum_ik v D_ik   -> K_jl and K_lj
// Blocks of up to 128 elements are digested by one thread each (a warp
// covers 32 quartets); larger blocks by one warp each, whose lanes own output
// entries of one contraction at a time (no two lanes add to the same entry).
// Blocks are read through L1; J and K receive FP64 reductions.
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
};

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
// share its output entries (W = 1: one thread does all of them).
template <int W>
__device__ __forceinline__ void eri_digest_quartet(const EriDigestArgs& g, int64_t q, int lane,
                                                   const double* __restrict__ v) {
  const int a = g.quartets[4 * q], b = g.quartets[4 * q + 1], c = g.quartets[4 * q + 2], d = g.quartets[4 * q + 3];
  const int A = g.shell_bf[a], B = g.shell_bf[b], C = g.shell_bf[c], Dd = g.shell_bf[d];
  const int na = g.shell_bf[a + 1] - A, nb = g.shell_bf[b + 1] - B, nc = g.shell_bf[c + 1] - C,
            nd = g.shell_bf[d + 1] - Dd;
  const double f = 1.0 / (double)eri_stabilizer(a, b, c, d);
  const double* __restrict__ Dm = g.D;
  const int64_t n = g.nbf;
  const int sj = nc * nd, si = nb * sj;  // strides of i and j in the block; k stride nd
  if (g.J) {
    // Jab[i][j] = 2 f sum_kl v D_kl
    for (int o = lane; o < na * nb; o += W) {
      const int i = o / nb, j = o - i * nb;
      const double* r = v + (int64_t)i * si + (int64_t)j * sj;
      double s = 0.0;
      for (int k = 0; k < nc; ++k)
        for (int l = 0; l < nd; ++l) s = fma(r[k * nd + l], __ldg(Dm + (C + k) * n + Dd + l), s);
      s *= 2.0 * f;
      atomicAdd(g.J + (A + i) * n + B + j, s);
      atomicAdd(g.J + (B + j) * n + A + i, s);
    }
    // Jcd[k][l] = 2 f sum_ij v D_ij
    for (int o = lane; o < nc * nd; o += W) {
      const int k = o / nd, l = o - k * nd;
      double s = 0.0;
      for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j)
          s = fma(v[(int64_t)i * si + (int64_t)j * sj + o], __ldg(Dm + (A + i) * n + B + j), s);
      s *= 2.0 * f;
      atomicAdd(g.J + (C + k) * n + Dd + l, s);
      atomicAdd(g.J + (Dd + l) * n + C + k, s);
    }
  }
  if (g.K) {
    // Kac[i][k] = f sum_jl v D_jl
    for (int o = lane; o < na * nc; o += W) {
      const int i = o / nc, k = o - i * nc;
      double s = 0.0;
      for (int j = 0; j < nb; ++j)
        for (int l = 0; l < nd; ++l)
          s = fma(v[(int64_t)i * si + (int64_t)j * sj + k * nd + l], __ldg(Dm + (B + j) * n + Dd + l), s);
      s *= f;
      atomicAdd(g.K + (A + i) * n + C + k, s);
      atomicAdd(g.K + (C + k) * n + A + i, s);
    }
    // Kad[i][l] = f sum_jk v D_jk
    for (int o = lane; o < na * nd; o += W) {
      const int i = o / nd, l = o - i * nd;
      double s = 0.0;
      for (int j = 0; j < nb; ++j)
        for (int k = 0; k < nc; ++k)
          s = fma(v[(int64_t)i * si + (int64_t)j * sj + k * nd + l], __ldg(Dm + (B + j) * n + C + k), s);
      s *= f;
      atomicAdd(g.K + (A + i) * n + Dd + l, s);
      atomicAdd(g.K + (Dd + l) * n + A + i, s);
    }
    // Kbc[j][k] = f sum_il v D_il
    for (int o = lane; o < nb * nc; o += W) {
      const int j = o / nc, k = o - j * nc;
      double s = 0.0;
      for (int i = 0; i < na; ++i)
        for (int l = 0; l < nd; ++l)
          s = fma(v[(int64_t)i * si + (int64_t)j * sj + k * nd + l], __ldg(Dm + (A + i) * n + Dd + l), s);
      s *= f;
      atomicAdd(g.K + (B + j) * n + C + k, s);
      atomicAdd(g.K + (C + k) * n + B + j, s);
    }
    // Kbd[j][l] = f sum_ik v D_ik
    for (int o = lane; o < nb * nd; o += W) {
      const int j = o / nd, l = o - j * nd;
      double s = 0.0;
      for (int i = 0; i < na; ++i)
        for (int k = 0; k < nc; ++k)
          s = fma(v[(int64_t)i * si + (int64_t)j * sj + k * nd + l], __ldg(Dm + (A + i) * n + C + k), s);
      s *= f;
      atomicAdd(g.K + (B + j) * n + Dd + l, s);
      atomicAdd(g.K + (Dd + l) * n + B + j, s);
    }
  }
}

__global__ void __launch_bounds__(128) eri_digest_small_kernel(const EriDigestArgs g) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < g.nlist) {
    const int64_t q = g.list[t];
    eri_digest_quartet<1>(g, q, 0, g.blocks + g.offsets[q]);
  }
}

__global__ void __launch_bounds__(128) eri_digest_warp_kernel(const EriDigestArgs g) {
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (w < g.nlist) {
    const int64_t q = g.list[w];
    eri_digest_quartet<32>(g, q, threadIdx.x & 31, g.blocks + g.offsets[q]);
  }
}

// small = 1: one thread per quartet of the list (32 per warp), else one warp
// per quartet
extern "C" cudaError_t eri_digest_launch(const EriDigestArgs* g, int small, cudaStream_t stream) {
  if (g->nlist == 0) return cudaSuccess;
  const int64_t grid = small ? (g->nlist + 127) / 128 : (g->nlist + 3) / 4;
  if (small)
    eri_digest_small_kernel<<<(unsigned)grid, 128, 0, stream>>>(*g);
  else
    eri_digest_warp_kernel<<<(unsigned)grid, 128, 0, stream>>>(*g);
  return cudaGetLastError();
}
