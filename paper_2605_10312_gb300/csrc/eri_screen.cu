// Schwarz screening of the unique shell-quartet list on the device.
//
// |(ab|cd)| <= Q_ab Q_cd with Q_ab = sqrt(max |(ab|ab)|) (the Cauchy-Schwarz
// inequality for the ERI inner product); the batched workload keeps the
// quartets whose bound reaches a threshold.  The unique quartets are the
// unordered pairs {P, R} of shell pairs (P = R included).  For P, R let lo
// be the one with the smaller factor (the larger index among equal
// factors) and hi the other: the quartet survives iff Q_hi >= t / Q_lo
// (for Q_lo = 0: iff t <= 0).  Phrased with the division, the rule picks
// the same set as the host's sorted-prefix enumeration, bit for bit.
//
// Three launches, all on the caller's stream:
//   1. count: one block per pair p counts its partners r <= p;
//   2. scan: one block turns the counts into output offsets (exclusive
//      prefix sum, the total in the last entry);
//   3. write: one block per pair p compacts its survivors (warp ballots and
//      a block-wide prefix of the warp counts) into out[offset[p] ...] as
//      (P.a, P.b, R.a, R.b) with P = pair p, in increasing r.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ bool eri_survives(double qp, double qr, int64_t p, int64_t r, double t) {
  // lo: smaller factor; among equal factors the larger index
  const bool p_lo = qp < qr || (qp == qr && p > r);
  const double lo = p_lo ? qp : qr, hi = p_lo ? qr : qp;
  return lo > 0.0 ? hi >= t / lo : t <= 0.0;
}

__global__ void __launch_bounds__(kThreads) eri_screen_count_kernel(const double* __restrict__ Q, int64_t npair,
                                                                    double t, int64_t* __restrict__ cnt) {
  __shared__ int64_t part[kThreads / 32];
  for (int64_t p = blockIdx.x; p < npair; p += gridDim.x) {
    const double qp = Q[p];
    int64_t c = 0;
    for (int64_t r = threadIdx.x; r <= p; r += kThreads) c += eri_survives(qp, __ldg(Q + r), p, r, t) ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t s = 0;
      for (int w = 0; w < kThreads / 32; ++w) s += part[w];
      cnt[p] = s;
    }
    __syncthreads();
  }
}

// Exclusive prefix sum of cnt[0..n) into off[0..n], off[n] = total; one block.
__global__ void __launch_bounds__(kThreads) eri_screen_scan_kernel(const int64_t* __restrict__ cnt, int64_t n,
                                                                   int64_t* __restrict__ off) {
  __shared__ int64_t warp_sum[kThreads / 32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = 0; base < n; base += kThreads) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < n ? cnt[i] : 0;
    int64_t x = v;  // inclusive scan within the warp
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    int64_t before = carry;
    for (int w = 0; w < warp; ++w) before += warp_sum[w];
    if (i < n) off[i] = before + x - v;
    __syncthreads();
    if (threadIdx.x == kThreads - 1) carry = before + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) off[n] = carry;
}

__global__ void __launch_bounds__(kThreads) eri_screen_write_kernel(const double* __restrict__ Q,
                                                                    const int2* __restrict__ pairs, int64_t npair,
                                                                    double t, const int64_t* __restrict__ off,
                                                                    int4* __restrict__ out) {
  __shared__ int warp_n[kThreads / 32];
  __shared__ int64_t written;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t p = blockIdx.x; p < npair; p += gridDim.x) {
    const double qp = Q[p];
    const int2 P = pairs[p];
    if (threadIdx.x == 0) written = 0;
    __syncthreads();
    for (int64_t base = 0; base <= p; base += kThreads) {
      const int64_t r = base + threadIdx.x;
      const bool keep = r <= p && eri_survives(qp, __ldg(Q + r), p, r, t);
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (lane == 0) warp_n[warp] = __popc(m);
      __syncthreads();
      int64_t at = written;
      for (int w = 0; w < warp; ++w) at += warp_n[w];
      at += __popc(m & ((1u << lane) - 1u));
      if (keep) {
        const int2 R = pairs[r];
        out[off[p] + at] = make_int4(P.x, P.y, R.x, R.y);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        int64_t s = 0;
        for (int w = 0; w < kThreads / 32; ++w) s += warp_n[w];
        written += s;
      }
      __syncthreads();
    }
  }
}

int screen_grid(int64_t npair) {
  int dev = 0, nsm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (int64_t)nsm * 8;  // eight 256-thread blocks per SM, striding over the pairs
  return (int)(npair < want ? npair : want);
}

}  // namespace

// Counts and offsets: off must hold npair + 1 entries, cnt npair.
extern "C" cudaError_t eri_screen_count_launch(const double* Q, int64_t npair, double t, int64_t* cnt, int64_t* off,
                                               cudaStream_t stream) {
  if (npair <= 0) return cudaSuccess;
  eri_screen_count_kernel<<<screen_grid(npair), kThreads, 0, stream>>>(Q, npair, t, cnt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  eri_screen_scan_kernel<<<1, kThreads, 0, stream>>>(cnt, npair, off);
  return cudaGetLastError();
}

extern "C" cudaError_t eri_screen_write_launch(const double* Q, const int32_t* pairs, int64_t npair, double t,
                                               const int64_t* off, int32_t* out, cudaStream_t stream) {
  if (npair <= 0) return cudaSuccess;
  eri_screen_write_kernel<<<screen_grid(npair), kThreads, 0, stream>>>(Q, reinterpret_cast<const int2*>(pairs), npair,
                                                                       t, off, reinterpret_cast<int4*>(out));
  return cudaGetLastError();
}
