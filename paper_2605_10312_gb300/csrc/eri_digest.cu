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
// Blocks are read through L1; J and K receive FP64 reductions.  With
// EriDigestArgs.tri the two mirrored entries of each contribution receive
// one reduction, into a triangle that is folded into J and K afterwards.
#include "eri_digest.cuh"

__global__ void __launch_bounds__(128) eri_digest_small_kernel(const EriDigestArgs g) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < g.nlist) {
    const int64_t q = g.list[t];
    eri_digest_quartet(g, q, 0, 1, g.blocks + g.offsets[q], [](const double* p) { return *p; });
  }
}

__global__ void __launch_bounds__(128) eri_digest_warp_kernel(const EriDigestArgs g) {
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (w < g.nlist) {
    const int64_t q = g.list[w];
    eri_digest_quartet(g, q, threadIdx.x & 31, 32, g.blocks + g.offsets[q], [](const double* p) { return *p; });
  }
}

// M[r][c] += T[min(r, c)][max(r, c)]: a triangle of mirrored-pair sums (see
// eri_jk_add) added into the caller's full n x n matrix.
__global__ void __launch_bounds__(256) eri_digest_fold_kernel(const double* __restrict__ T, double* __restrict__ M,
                                                             int n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int64_t r = t / n, c = t - r * n;
  M[t] += r <= c ? T[t] : T[c * n + r];
}

extern "C" cudaError_t eri_digest_fold_launch(const double* T, double* M, int n, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int64_t nn = (int64_t)n * n;
  eri_digest_fold_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, stream>>>(T, M, n);
  return cudaGetLastError();
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
