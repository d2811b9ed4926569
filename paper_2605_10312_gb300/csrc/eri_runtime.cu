// Runtime behind the C ABI of include/eri.h: plan construction (validation,
// per-quartet canonicalisation and orientation, shell-pair deduplication,
// class bucketing, tier routing, device upload) and eri_compute (the pair
// set-up kernel followed by one launch per class bucket).
//
// Class programs and the Boys table come from the generator's blob
// (eri_programs*.bin next to this library); register-tier kernels are linked
// in through the generated registry.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "eri.h"
#include "eri_common.cuh"
#include "eri_coop.cuh"
#include "eri_digest.cuh"

// ---------------------------------------------------------------------------
// executor and registry (other translation units)
// ---------------------------------------------------------------------------
extern "C" cudaError_t eri_exec_launch(int shared, const EriLaunchArgs* a, const EriProgArgs* p, int grid,
                                       int block, size_t smem, cudaStream_t stream);
extern "C" cudaError_t eri_exec_set_smem(size_t bytes);
extern "C" cudaError_t eri_exec_boys_launch(const double* T, int64_t n, int L, const double* tab, double* F,
                                            cudaStream_t stream);
extern "C" cudaError_t eri_coop_boys_launch(const double* T, int64_t n, int L, const double* tab, double* F,
                                            cudaStream_t stream);

extern "C" cudaError_t eri_digest_launch(const EriDigestArgs* g, int small, cudaStream_t stream);
extern "C" cudaError_t eri_digest_fold_launch(const double* T, double* M, int n, cudaStream_t stream);
// blocks of up to this many elements are digested by one thread each
static const int64_t kSmallBlock = 128;

extern "C" cudaError_t eri_coop_launch(int T, int ilp, int fp32, int vote, const EriLaunchArgs* a,
                                       const EriCoopArgs* p, int grid, int block, size_t smem, cudaStream_t stream);
extern "C" cudaError_t eri_coop_set_smem(size_t bytes);
extern "C" cudaError_t eri_coop_persist_launch(int fp32, int vote, const EriLaunchArgs* a, const EriPersistArgs* pa,
                                               int grid, size_t smem, cudaStream_t stream);
extern "C" size_t eri_coop_persist_smem_max(size_t optin);
extern "C" size_t eri_coop_row_elems(void);
extern "C" int eri_coop_max_batch(void);
// contractions of at most this many primitive quartets per part use the
// cooperative tier's shallow-contraction shape (the generator's SHALLOW_ROWS)
static const int kShallowK4 = 12;

struct EriRegEntry {
  int8_t ls[4];
  const void* fn;
};
extern "C" const EriRegEntry eri_reg_table[];
extern "C" const int eri_reg_count;
extern "C" const EriRegEntry eri_reg_f32_table[];  // FP32-recurrence forms
extern "C" const int eri_reg_f32_count;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CUDA_OR(expr, what)                                                               \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess) return fail(ERI_ECUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
  } while (0)

extern "C" const char* eri_last_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------------------
// program blob
// ---------------------------------------------------------------------------
namespace {

struct ClassProg {
  int ls[4];
  int opts[3];  // axis rule, schedule, sph mode
  int nh, nslot, L, n1, n2, kmax;
  int dims[4];
  double flops_prim, flops_p2;
  std::vector<uint32_t> ph1, ph2;
  // device copies (lazily uploaded)
  uint4* d_ph1 = nullptr;
  uint4* d_ph2 = nullptr;
};

struct CoopProg {
  int ls[4];
  int opts[3];
  int ilp;
  int T, nh, nslot, L, nw1, nw2, n1, n2;
  int k1 = 1, k2 = 1;  // steps per Phase-1 / Phase-2 wave
  int dims[4];
  double flops_prim, flops_p2;
  std::vector<uint32_t> steps1, steps2, ph1, ph2;
  uint32_t* d_steps1 = nullptr;
  uint32_t* d_steps2 = nullptr;
  uint4* d_ph1 = nullptr;
  uint4* d_ph2 = nullptr;
};

struct Library {
  bool loaded = false;
  std::string err;
  std::vector<double> boys, c2s;
  std::map<std::vector<int>, std::unique_ptr<ClassProg>> progs;  // key: ls[4] + opts[3]
  std::map<std::vector<int>, std::unique_ptr<CoopProg>> coops;   // key: ls[4] + opts[3]
  std::map<std::vector<int>, std::unique_ptr<CoopProg>> coops_shallow;  // shapes for K4 <= kShallowK4
  std::map<std::vector<int>, std::vector<std::unique_ptr<CoopProg>>> coops_alt;  // autotuner candidates
  std::map<std::vector<int>, const void*> reg;                      // key: ls[4]
  std::map<std::vector<int>, const void*> reg_f32;                  // key: ls[4]
  double* d_boys = nullptr;
  double* d_c2s = nullptr;
  int device = -1;
  int nsm = 0;
  size_t smem_optin = 0;
  size_t smem_per_sm = 0;
  std::mutex mu;
};

Library& lib() {
  static Library L;
  return L;
}

std::string lib_dir() {
  Dl_info info;
  if (dladdr((void*)&eri_last_error, &info) && info.dli_fname) {
    std::string p(info.dli_fname);
    size_t k = p.rfind('/');
    return k == std::string::npos ? std::string(".") : p.substr(0, k);
  }
  return ".";
}

template <typename T>
bool rd(FILE* f, T* v, size_t n = 1) {
  return fread(v, sizeof(T), n, f) == n;
}

bool load_blob(Library& L, const std::string& path, bool tables) {
  FILE* f = fopen(path.c_str(), "rb");
  if (!f) return false;
  char magic[8];
  uint32_t nb = 0, nc = 0, ncls = 0;
  bool ok = rd(f, magic, 8) && memcmp(magic, "ERIPRG03", 8) == 0 && rd(f, &nb);
  std::vector<double> boys(nb);
  ok = ok && rd(f, boys.data(), nb) && rd(f, &nc);
  std::vector<double> c2s(nc);
  ok = ok && rd(f, c2s.data(), nc) && rd(f, &ncls);
  for (uint32_t c = 0; ok && c < ncls; ++c) {
    auto p = std::make_unique<ClassProg>();
    int8_t hdr[8];
    int32_t iv[10];
    double fv[2];
    ok = rd(f, hdr, 8) && rd(f, iv, 10) && rd(f, fv, 2);
    if (!ok) break;
    for (int k = 0; k < 4; ++k) p->ls[k] = hdr[k];
    for (int k = 0; k < 3; ++k) p->opts[k] = hdr[4 + k];
    p->nh = iv[0];
    p->nslot = iv[1];
    p->L = iv[2];
    p->n1 = iv[3];
    p->n2 = iv[4];
    p->kmax = iv[5];
    for (int k = 0; k < 4; ++k) p->dims[k] = iv[6 + k];
    p->flops_prim = fv[0];
    p->flops_p2 = fv[1];
    p->ph1.resize((size_t)p->n1 * 4);
    p->ph2.resize((size_t)p->n2 * 4);
    ok = rd(f, p->ph1.data(), p->ph1.size()) && rd(f, p->ph2.data(), p->ph2.size());
    if (!ok) break;
    std::vector<int> key = {p->ls[0], p->ls[1], p->ls[2], p->ls[3], p->opts[0], p->opts[1], p->opts[2]};
    L.progs[key] = std::move(p);
  }
  // team-cooperative programs: the deep-contraction section, the
  // shallow-contraction section (shapes that differ from the deep one), then
  // the autotuner's alternative shapes
  for (int section = 0; section < 3 && ok; ++section) {
    uint32_t ncoop = 0;
    if (!rd(f, &ncoop)) break;
    for (uint32_t c = 0; ok && c < ncoop; ++c) {
      auto p = std::make_unique<CoopProg>();
      int8_t hdr[8];
      int32_t iv[15];
      double fv[2];
      ok = rd(f, hdr, 8) && rd(f, iv, 15) && rd(f, fv, 2);
      if (!ok) break;
      for (int k = 0; k < 4; ++k) p->ls[k] = hdr[k];
      for (int k = 0; k < 3; ++k) p->opts[k] = hdr[4 + k];
      p->ilp = hdr[7] ? hdr[7] : 2;
      if (iv[12] != 1) ok = false;  // full-barrier programs only
      p->T = iv[0];
      p->nh = iv[1];
      p->nslot = iv[2];
      p->L = iv[3];
      p->nw1 = iv[4];
      p->nw2 = iv[5];
      p->n1 = iv[6];
      p->n2 = iv[7];
      for (int k = 0; k < 4; ++k) p->dims[k] = iv[8 + k];
      p->k1 = iv[13];
      p->k2 = iv[14];
      p->flops_prim = fv[0];
      p->flops_p2 = fv[1];
      p->steps1.resize(p->nw1);
      p->steps2.resize(p->nw2);
      p->ph1.resize((size_t)p->n1 * 4);
      p->ph2.resize((size_t)p->n2 * 4);
      ok = rd(f, p->steps1.data(), p->steps1.size()) && rd(f, p->steps2.data(), p->steps2.size()) &&
           rd(f, p->ph1.data(), p->ph1.size()) && rd(f, p->ph2.data(), p->ph2.size());
      if (!ok) break;
      std::vector<int> key = {p->ls[0], p->ls[1], p->ls[2], p->ls[3], p->opts[0], p->opts[1], p->opts[2]};
      if (section == 2)
        L.coops_alt[key].push_back(std::move(p));
      else
        (section == 0 ? L.coops : L.coops_shallow)[key] = std::move(p);
    }
  }
  fclose(f);
  if (ok && tables) {
    L.boys = boys;
    L.c2s = c2s;
  }
  return ok;
}

int ensure_library() {
  Library& L = lib();
  std::lock_guard<std::mutex> g(L.mu);
  int dev = 0;
  CUDA_OR(cudaGetDevice(&dev), "cudaGetDevice");
  if (!L.loaded) {
    std::string dir = lib_dir();
    if (!load_blob(L, dir + "/eri_programs.bin", true))
      return fail(ERI_ESTATE, "cannot read " + dir + "/eri_programs.bin (run the build)");
    for (const char* extra : {"/eri_programs_ablation.bin"}) load_blob(L, dir + extra, false);
    for (int i = 0; i < eri_reg_count; ++i) {
      const EriRegEntry& e = eri_reg_table[i];
      L.reg[{e.ls[0], e.ls[1], e.ls[2], e.ls[3]}] = e.fn;
    }
    for (int i = 0; i < eri_reg_f32_count; ++i) {
      const EriRegEntry& e = eri_reg_f32_table[i];
      L.reg_f32[{e.ls[0], e.ls[1], e.ls[2], e.ls[3]}] = e.fn;
    }
    L.loaded = true;
  }
  if (L.device != dev) {
    if (L.device >= 0) return fail(ERI_EUNSUPPORTED, "the library serves one CUDA device per process");
    CUDA_OR(cudaMalloc(&L.d_boys, L.boys.size() * sizeof(double)), "cudaMalloc boys table");
    CUDA_OR(cudaMemcpy(L.d_boys, L.boys.data(), L.boys.size() * sizeof(double), cudaMemcpyHostToDevice),
            "upload boys table");
    CUDA_OR(cudaMalloc(&L.d_c2s, std::max<size_t>(1, L.c2s.size()) * sizeof(double)), "cudaMalloc c2s");
    CUDA_OR(cudaMemcpy(L.d_c2s, L.c2s.data(), L.c2s.size() * sizeof(double), cudaMemcpyHostToDevice),
            "upload c2s");
    cudaDeviceProp prop;
    CUDA_OR(cudaGetDeviceProperties(&prop, dev), "cudaGetDeviceProperties");
    L.nsm = prop.multiProcessorCount;
    L.smem_optin = prop.sharedMemPerBlockOptin;
    L.smem_per_sm = prop.sharedMemPerMultiprocessor;
    CUDA_OR(eri_exec_set_smem(L.smem_optin), "cudaFuncSetAttribute");
    CUDA_OR(eri_coop_set_smem(L.smem_optin), "cudaFuncSetAttribute");
    L.device = dev;
  }
  return ERI_OK;
}

int upload_prog(ClassProg* p) {
  Library& L = lib();
  std::lock_guard<std::mutex> g(L.mu);
  if (p->d_ph1) return ERI_OK;
  CUDA_OR(cudaMalloc(&p->d_ph1, std::max<size_t>(1, p->ph1.size()) * 4), "cudaMalloc program");
  CUDA_OR(cudaMalloc(&p->d_ph2, std::max<size_t>(1, p->ph2.size()) * 4), "cudaMalloc program");
  CUDA_OR(cudaMemcpy(p->d_ph1, p->ph1.data(), p->ph1.size() * 4, cudaMemcpyHostToDevice), "upload program");
  CUDA_OR(cudaMemcpy(p->d_ph2, p->ph2.data(), p->ph2.size() * 4, cudaMemcpyHostToDevice), "upload program");
  return ERI_OK;
}

int upload_coop(CoopProg* p) {
  Library& L = lib();
  std::lock_guard<std::mutex> g(L.mu);
  if (p->d_ph1) return ERI_OK;
  CUDA_OR(cudaMalloc(&p->d_steps1, std::max<size_t>(1, p->steps1.size()) * 4), "cudaMalloc program");
  CUDA_OR(cudaMalloc(&p->d_steps2, std::max<size_t>(1, p->steps2.size()) * 4), "cudaMalloc program");
  CUDA_OR(cudaMalloc(&p->d_ph1, std::max<size_t>(1, p->ph1.size()) * 4), "cudaMalloc program");
  CUDA_OR(cudaMalloc(&p->d_ph2, std::max<size_t>(1, p->ph2.size()) * 4), "cudaMalloc program");
  CUDA_OR(cudaMemcpy(p->d_steps1, p->steps1.data(), p->steps1.size() * 4, cudaMemcpyHostToDevice), "upload");
  CUDA_OR(cudaMemcpy(p->d_steps2, p->steps2.data(), p->steps2.size() * 4, cudaMemcpyHostToDevice), "upload");
  CUDA_OR(cudaMemcpy(p->d_ph1, p->ph1.data(), p->ph1.size() * 4, cudaMemcpyHostToDevice), "upload");
  CUDA_OR(cudaMemcpy(p->d_ph2, p->ph2.data(), p->ph2.size() * 4, cudaMemcpyHostToDevice), "upload");
  return ERI_OK;
}

// ---------------------------------------------------------------------------
// device data the pair set-up kernel consumes
// ---------------------------------------------------------------------------
struct DevShell {
  double ctr[3];
  int32_t l, nprim, prim;
  int32_t pad;
};
struct DevPairIn {
  int32_t a, b;       // oriented shells: a is the recurrence centre
  int32_t prim_off;   // first EriPairPrim
  int32_t list_off;   // -1: every (i, j) of a x b; -2: alias of nlist primitive pairs already
                      // written at prim_off (a chunk of another pair); else nlist packed
                      // (i | j << 16) entries of the primitive-pair list
  int32_t nlist;
  int32_t pad;
};

// uint64 -> int32 hash map with open addressing (linear probing): the plan's
// pair, split, alias and signature tables see one lookup per quartet part.
class FlatMap {
 public:
  explicit FlatMap(size_t expect = 16) { rehash(cap_for(expect)); }
  // index of key, inserting make() when absent
  template <typename Make>
  int32_t get_or_insert(uint64_t key, Make make) {
    if (2 * (size_ + 1) > keys_.size()) rehash(keys_.size() * 2);
    size_t i = slot(key);
    while (keys_[i] != kEmpty) {
      if (keys_[i] == key) return vals_[i];
      i = (i + 1) & (keys_.size() - 1);
    }
    const int32_t v = make();
    keys_[i] = key;
    vals_[i] = v;
    ++size_;
    return v;
  }
  // value of key, or -1
  int32_t find(uint64_t key) const {
    size_t i = slot(key);
    while (keys_[i] != kEmpty) {
      if (keys_[i] == key) return vals_[i];
      i = (i + 1) & (keys_.size() - 1);
    }
    return -1;
  }

 private:
  static constexpr uint64_t kEmpty = ~(uint64_t)0;
  std::vector<uint64_t> keys_;
  std::vector<int32_t> vals_;
  size_t size_ = 0;
  static size_t cap_for(size_t n) {
    size_t c = 16;
    while (c < 2 * n) c <<= 1;
    return c;
  }
  size_t slot(uint64_t k) const {
    k += 0x9e3779b97f4a7c15ull;  // splitmix64 finaliser
    k = (k ^ (k >> 30)) * 0xbf58476d1ce4e5b9ull;
    k = (k ^ (k >> 27)) * 0x94d049bb133111ebull;
    k ^= k >> 31;
    return (size_t)k & (keys_.size() - 1);
  }
  void rehash(size_t cap) {
    std::vector<uint64_t> ok;
    std::vector<int32_t> ov;
    ok.swap(keys_);
    ov.swap(vals_);
    keys_.assign(cap, kEmpty);
    vals_.assign(cap, 0);
    size_ = 0;
    for (size_t i = 0; i < ok.size(); ++i)
      if (ok[i] != kEmpty) get_or_insert(ok[i], [&] { return ov[i]; });
  }
};

// An oriented (partial) shell pair of a quartet: the pair record `pair`
// recurs on shell `center`, with `nprim` primitive pairs.
struct PairPart {
  int center, other, pair, nprim;
};
struct SplitRes {
  int n;
  PairPart part[2];
};

// Shell pairs in recurrence orientation, and the list the pair set-up
// kernel consumes (one DevPairIn per oriented partial pair).
//   orientation 0: each primitive pair recurs on its tighter primitive's
//   centre, so a contracted pair splits into at most two oriented partial
//   pairs (kind 1: primitive pairs whose centre exponent is >= the other's,
//   kind 2: > the other's); this keeps FP64 HRR cancellation bounded;
//   orientation 1: the whole pair on the higher l; 2: on the shell holding
//   the largest exponent.  Kind 0 = every primitive pair.
struct PairBuilder {
  const eri_shell* shells;
  const eri_basis* basis;
  const std::vector<double>* maxexp;
  int orientation;
  FlatMap pair_id;
  std::vector<DevPairIn> pin;
  std::vector<uint32_t> plist;
  int64_t pprim = 0;

  int get_pair(int a, int b, int kind) {
    const uint64_t key = ((uint64_t)(uint32_t)a << 34) | ((uint64_t)(uint32_t)b << 2) | (uint64_t)kind;
    return pair_id.get_or_insert(key, [&] { return make_pair(a, b, kind); });
  }

  int make_pair(int a, int b, int kind) {
    int id = (int)pin.size();
    DevPairIn d{a, b, (int32_t)pprim, -1, 0, 0};
    if (kind == 0) {
      pprim += (int64_t)shells[a].nprim * shells[b].nprim;
    } else {
      d.list_off = (int32_t)plist.size();
      const double* ea = basis->exponents + shells[a].prim_offset;
      const double* eb = basis->exponents + shells[b].prim_offset;
      for (int i = 0; i < shells[a].nprim; ++i)
        for (int j = 0; j < shells[b].nprim; ++j)
          if (kind == 1 ? ea[i] >= eb[j] : ea[i] > eb[j]) plist.push_back((uint32_t)i | ((uint32_t)j << 16));
      d.nlist = (int32_t)plist.size() - d.list_off;
      pprim += d.nlist;
    }
    pin.push_back(d);
    return id;
  }

  // the oriented parts of shell pair (s0, s1); callers pass s0 >= s1 so that
  // ties between equal exponents of different shells break the same way
  int split(int s0, int s1, PairPart* out) {
    const int l0 = shells[s0].l, l1 = shells[s1].l;
    if (orientation == 1 || orientation == 2) {
      const std::vector<double>& mx = *maxexp;
      bool first = orientation == 1 ? l0 >= l1 : (mx[s0] != mx[s1] ? mx[s0] > mx[s1] : l0 >= l1);
      const int c = first ? s0 : s1, o = first ? s1 : s0;
      out[0] = {c, o, get_pair(c, o, 0), shells[s0].nprim * shells[s1].nprim};
      return 1;
    }
    const double* e0 = basis->exponents + shells[s0].prim_offset;
    const double* e1 = basis->exponents + shells[s1].prim_offset;
    int n0 = 0, n1 = 0;  // primitive pairs recurring on s0 / on s1
    for (int i = 0; i < shells[s0].nprim; ++i)
      for (int j = 0; j < shells[s1].nprim; ++j) (e0[i] >= e1[j] ? n0 : n1)++;
    int k = 0;
    if (n1 == 0) {
      out[k++] = {s0, s1, get_pair(s0, s1, 0), n0};
    } else if (n0 == 0) {
      out[k++] = {s1, s0, get_pair(s1, s0, 0), n1};
    } else {
      out[k++] = {s0, s1, get_pair(s0, s1, 1), n0};
      out[k++] = {s1, s0, get_pair(s1, s0, 2), n1};
    }
    return k;
  }
};

}  // namespace

// FusionRCG Algorithm 2, "GaussianPairs", once per primitive pair: zeta,
// P, P - A, and the pair factor sqrt(2) pi^(5/4) c_a N_a c_b N_b
// exp(-a b |A-B|^2 / zeta) / zeta, so that the primitive-quartet prefactor
// 2 pi^(5/2) / (zeta eta sqrt(zeta+eta)) K_AB K_CD is one product.
__global__ void eri_pair_setup_kernel(const DevPairIn* __restrict__ pin, int npair, const DevShell* __restrict__ sh,
                                      const double* __restrict__ ex, const double* __restrict__ co,
                                      const uint32_t* __restrict__ plist, EriPairRec* __restrict__ pairs,
                                      EriPairPrim* __restrict__ pp, EriPairPrimF* __restrict__ ppf) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npair) return;
  const DevPairIn in = pin[p];
  const DevShell A = sh[in.a], B = sh[in.b];
  const double AB0 = A.ctr[0] - B.ctr[0], AB1 = A.ctr[1] - B.ctr[1], AB2 = A.ctr[2] - B.ctr[2];
  const double ab2 = AB0 * AB0 + AB1 * AB1 + AB2 * AB2;
  EriPairRec r;
  r.prim_off = in.prim_off;
  const int n = in.list_off == -1 ? A.nprim * B.nprim : in.nlist;
  r.nprim = n;
  r.AB[0] = AB0;
  r.AB[1] = AB1;
  r.AB[2] = AB2;
  pairs[p] = r;
  if (in.list_off == -2) return;  // a chunk: its primitive pairs belong to another record
  const double dfi[5] = {1.0, 1.0, 1.0 / 1.7320508075688772935, 1.0 / 3.8729833462074168852,
                         1.0 / 10.246950765959598383};  // 1/sqrt((2l-1)!!)
  const double C0 = 5.9149671727956128778;              // sqrt(2) pi^(5/4)
  for (int k = 0; k < n; ++k) {
    int i, j;
    if (in.list_off < 0) {
      i = k / B.nprim;
      j = k - i * B.nprim;
    } else {
      const uint32_t e = plist[in.list_off + k];
      i = (int)(e & 0xFFFF);
      j = (int)(e >> 16);
    }
    const double a = ex[A.prim + i];
    const double xa = a * 0.63661977236758134308;  // 2a/pi
    double na = sqrt(xa * sqrt(xa)) * dfi[A.l];
    const double sa = sqrt(4.0 * a);
    for (int t = 0; t < A.l; ++t) na *= sa;
    const double b = ex[B.prim + j];
    const double xb = b * 0.63661977236758134308;
    double nb = sqrt(xb * sqrt(xb)) * dfi[B.l];
    const double sb = sqrt(4.0 * b);
    for (int t = 0; t < B.l; ++t) nb *= sb;
    const double z = a + b;
    const double iz = 1.0 / z;
    EriPairPrim q;
    q.zeta = z;
    q.inv2z = 0.5 * iz;
    for (int d = 0; d < 3; ++d) {
      q.P[d] = (a * A.ctr[d] + b * B.ctr[d]) * iz;
      q.PA[d] = q.P[d] - A.ctr[d];
    }
    q.K = C0 * co[A.prim + i] * na * co[B.prim + j] * nb * exp(-a * b * iz * ab2) * iz;
    pp[in.prim_off + k] = q;
    if (ppf) ppf[in.prim_off + k] = eri_pair_prim_f32(q);
  }
}

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
namespace {
enum Tier { TIER_REG = 1, TIER_SHARED = 2, TIER_GLOBAL = 3, TIER_COOP = 4, TIER_PERSIST = 5 };

struct Bucket {
  int ls[4];
  int tier;
  const void* reg_fn = nullptr;
  ClassProg* prog = nullptr;
  int64_t first = 0, count = 0;  // range in the sorted quartet records
  int grid = 0, block = 128;
  size_t smem = 0;
  int group = 1;                 // lanes per shell quartet
  double flops = 0;              // algorithmic FP64 flops of this launch
  CoopProg* coop = nullptr;      // team-cooperative tier
  int smem_slots = 0, h_in_smem = 0, nteams = 0;
  int batch = 0;                 // cooperative tier: coefficient rows per team
  int single = 0;                // cooperative tier: every part has one primitive quartet
  int vote = 0;                  // cooperative tier: optional FP64 terms behind warp votes
  int kind = -1;                 // cooperative tier: 0 deep, 1 shallow, 2 single-primitive parts
  int shape = -1;                // cooperative tier: index of its program in class_shapes
  int fp32 = 0;                  // recurrences in FP32 (quartets with a small Schwarz bound)
  int round = 0;                 // part round: buckets of a round are independent
  int lane = 0;                  // stream of its round (0 = the caller's stream)
  bool shared_scratch = false;   // uses the plan's global scratch (runs on lane 0)
  // persistent plans: launch `pgroup` runs items [item0, item0 + nitems)
  int pgroup = -1, item0 = 0, nitems = 0;
};

// Plans built by eri_plan_on_stream allocate stream-ordered on that stream
// (set for the duration of the build on the building thread).
thread_local cudaStream_t g_alloc_stream = nullptr;
thread_local bool g_alloc_async = false;
struct AllocStreamScope {
  AllocStreamScope(cudaStream_t s, bool on) {
    g_alloc_stream = s;
    g_alloc_async = on;
  }
  ~AllocStreamScope() {
    g_alloc_stream = nullptr;
    g_alloc_async = false;
  }
};

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t st = nullptr;  // stream-ordered buffer (plans built on a stream), else nullptr
  bool async = false;
  ~DevBuf() { reset(); }
  void reset() {
    if (p) {
      if (async)
        cudaFreeAsync(p, st);
      else
        cudaFree(p);
    }
    p = nullptr;
    n = 0;
  }
  int alloc(size_t count, const char* what) {
    n = count;
    async = g_alloc_async;
    st = g_alloc_stream;
    if (count == 0) return ERI_OK;
    const cudaError_t e = async ? cudaMallocAsync((void**)&p, count * sizeof(T), st)
                                : cudaMalloc((void**)&p, count * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return fail(ERI_ENOMEM, std::string("device allocation failed: ") + what);
    }
    return ERI_OK;
  }
  int upload(const std::vector<T>& v, const char* what) {
    int rc = alloc(v.size(), what);
    if (rc) return rc;
    if (!v.empty()) {
      // pageable source: the copy is staged before the call returns
      if (async)
        CUDA_OR(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st), what);
      else
        CUDA_OR(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), what);
    }
    return ERI_OK;
  }
};
}  // namespace

// A molecule kept on the device (eri_mol_create): its shells, and every
// shell pair (a >= b) in recurrence orientation with its primitive-pair
// records computed once by the pair set-up kernel.
struct eri_mol_s {
  std::vector<eri_shell> shells;
  std::vector<double> centers, exps, coefs, maxexp;
  eri_basis view;                 // the vectors above as an eri_basis
  int nshell = 0;
  int orientation = 0;
  PairBuilder pb{nullptr, nullptr, nullptr, 0, FlatMap(), {}, {}, 0};
  std::vector<SplitRes> splits;   // per shell pair a >= b, at a (a + 1) / 2 + b
  int npair = 0;                  // oriented partial pairs (records)
  DevBuf<DevShell> shells_d;
  DevBuf<double> exps_d, coefs_d;
  DevBuf<DevPairIn> pin_d;
  DevBuf<uint32_t> plist_d;
  DevBuf<EriPairRec> pairs_d;
  DevBuf<EriPairPrim> pprims_d;
  DevBuf<EriPairPrimF> pprims_f;  // FP32 copy, for mixed-precision plans
};

struct eri_plan_s {
  const eri_mol_s* mol = nullptr;  // molecule plans: pairs and primitive pairs of the molecule
  int64_t nq = 0;
  std::vector<int64_t> offsets;  // nq + 1
  std::vector<Bucket> buckets;
  int npair = 0;
  int64_t npprim = 0;
  double flops = 0, nprimq = 0;
  double flops32 = 0;            // FP32 flops of the reduced-precision buckets
  int64_t nparts32 = 0;          // quartet parts evaluated with FP32 recurrences
  DevBuf<DevShell> shells;
  DevBuf<double> exps, coefs;
  DevBuf<DevPairIn> pin;
  DevBuf<uint32_t> plist;
  DevBuf<EriPairRec> pairs;
  DevBuf<EriPairPrim> pprims;
  DevBuf<EriPairPrimF> pprims_f;  // FP32 copy, when the plan has FP32 parts
  DevBuf<EriQuartetRec> quartets;
  DevBuf<double> scratch;
  DevBuf<double> outbuf;
  DevBuf<double> coop_vals, coop_h;  // team-private spill regions of the cooperative tier
  // persistent plans (eri_opts.persistent): work items, class programs, one
  // item counter per launch, the team-private H pool
  bool persistent = false;
  DevBuf<EriWorkItem> items;
  DevBuf<EriCoopProgDesc> progs;
  DevBuf<int32_t> counters;
  DevBuf<double> persist_h;
  int64_t persist_h_per_block = 0;
  DevBuf<int32_t> rec_q, nparts_q, done_q;  // fused digestion: record -> quartet, parts, finished parts
  int64_t scratch_stride = 0;
  double h2d_bytes = 0;
  bool zero_out = false;  // chunks reduce into their block: eri_compute zeroes the output first
  std::vector<int32_t> nab;          // (ab|ab) plans: components of ab per quartet (else empty)
  DevBuf<int64_t> d_offsets;         // block offsets, for (ab|ab) and digest plans
  DevBuf<int32_t> d_uq;              // digest plans: the caller's quartet list
  DevBuf<int32_t> d_shell_bf;        // digest plans: first basis function of each shell, and the total
  DevBuf<int64_t> d_small, d_large;  // digest plans: quartets with small / large blocks
  DevBuf<int64_t> d_rsmall, d_rlarge;  // fused digestion: the same lists for quartets with no persistent part
  int32_t nbf = 0;
  bool digest = false;
  DevBuf<double> jk_tri;             // digest plans: J and K triangles of mirrored-pair sums (2 nbf^2)
  DevBuf<int32_t> d_nab;
  cudaGraphExec_t graph_exec = nullptr;
  bool stream_ordered = false;         // built by eri_plan_on_stream: memory is freed on alloc_stream
  cudaStream_t alloc_stream = nullptr;
  int nlanes = 1;                      // streams one round's launches may use
  std::vector<cudaStream_t> lanes;     // lanes[k - 1] = stream of lane k >= 1 (plan-owned)
  cudaEvent_t fork_ev = nullptr;       // caller stream -> lanes
  std::vector<cudaEvent_t> join_ev;    // lane -> caller stream
  bool timing = false;
  std::vector<cudaEvent_t> events;  // two per launch: pair set-up, then buckets
  ~eri_plan_s() {
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    for (cudaEvent_t e : join_ev) cudaEventDestroy(e);
    if (fork_ev) cudaEventDestroy(fork_ev);
    for (cudaStream_t s : lanes) cudaStreamDestroy(s);
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
  }
};

static int nfun(int l, bool cart) { return cart ? (l + 1) * (l + 2) / 2 : 2 * l + 1; }
int preferred_tier(const int ls[4]);
int preferred_votes(const int ls[4]);
bool preferred_shape(const int ls[4], int kind, int* shape, int* votes);

// The cooperative shapes shipped for a class (default options): the deep
// shape, the shallow one when it differs, then the alternatives.  The index
// into this list names a shape in eri_class_shapes / eri_set_class_shape.
std::vector<CoopProg*> class_shapes(Library& L, const std::vector<int>& key) {
  std::vector<CoopProg*> v;
  auto d = L.coops.find(key);
  if (d == L.coops.end()) return v;
  v.push_back(d->second.get());
  auto sh = L.coops_shallow.find(key);
  if (sh != L.coops_shallow.end()) v.push_back(sh->second.get());
  auto al = L.coops_alt.find(key);
  if (al != L.coops_alt.end())
    for (auto& p : al->second) v.push_back(p.get());
  return v;
}

static int plan_impl(const eri_shell* shells, int32_t nshell, const eri_basis* basis, const int32_t* quartets,
                     int64_t nq, const double* qbound, double fp32_below, const eri_opts* opts_in,
                     eri_plan_t** plan_out, const eri_mol_s* mol = nullptr) {
  if (!plan_out) return fail(ERI_EINVAL, "plan_out is NULL");
  *plan_out = nullptr;
  eri_opts opts;
  memset(&opts, 0, sizeof opts);
  if (opts_in) opts = *opts_in;
  if (opts.axis_rule < 0 || opts.axis_rule > 2 || opts.schedule < 0 || opts.schedule > 1 || opts.sph_mode < 0 ||
      opts.sph_mode > 2 || opts.tier < 0 || opts.tier > 4 || opts.orientation < 0 || opts.orientation > 2 ||
      opts.streams < 0 || opts.streams > 8 || opts.digest < 0 || opts.digest > 1 || opts.votes < 0 ||
      opts.votes > 2 || opts.persistent < 0 || opts.persistent > 1 || opts.ordered < 0 || opts.ordered > 1)
    return fail(ERI_EINVAL, "option out of range");
  if (mol) {
    shells = mol->shells.data();
    nshell = mol->nshell;
    basis = &mol->view;
    if (opts.orientation != mol->orientation) return fail(ERI_EINVAL, "orientation differs from the molecule's");
  }
  if (nq < 0 || nshell < 0 || (nq > 0 && (!shells || !basis || !quartets)))
    return fail(ERI_EINVAL, "NULL or negative argument");
  // launches take their quartet count as int32
  if (nq > ((int64_t)1 << 31) - 1) return fail(ERI_EINVAL, "too many quartets for one plan (at most 2^31 - 1)");
  const bool cart = opts.sph_mode == 2;
  // persistent plans run every class on the team-cooperative programs
  if (opts.persistent && opts.tier != 0 && opts.tier != TIER_COOP)
    return fail(ERI_EINVAL, "a persistent plan takes tier 0 or 4");
  if (opts.persistent && opts.ordered) return fail(ERI_EINVAL, "a persistent plan reduces parts in any order");
  const bool persistent = opts.persistent == 1;
  // ---- validation
  if (nshell > 0) {
    if (!basis->centers || !basis->exponents || !basis->coefs || basis->ncenter < 0 || basis->nprim_total < 0)
      return fail(ERI_EINVAL, "incomplete basis");
  }
  std::vector<double> maxexp(nshell, 0.0);
  for (int s = 0; s < nshell; ++s) {
    const eri_shell& S = shells[s];
    if (S.l < 0) return fail(ERI_EINVAL, "shell " + std::to_string(s) + ": negative l");
    if (S.l > ERI_MAX_L) return fail(ERI_EUNSUPPORTED, "shell " + std::to_string(s) + ": l > 4");
    if (S.nprim < 1 || S.nprim > ERI_MAX_NPRIM) return fail(ERI_EINVAL, "shell " + std::to_string(s) + ": bad nprim");
    if (S.center < 0 || S.center >= basis->ncenter) return fail(ERI_EINVAL, "shell " + std::to_string(s) + ": bad centre");
    if (S.prim_offset < 0 || (int64_t)S.prim_offset + S.nprim > basis->nprim_total)
      return fail(ERI_EINVAL, "shell " + std::to_string(s) + ": primitives out of range");
    for (int k = 0; k < S.nprim; ++k) {
      const double a = basis->exponents[S.prim_offset + k], c = basis->coefs[S.prim_offset + k];
      if (!(a > 0) || !std::isfinite(a) || !std::isfinite(c))
        return fail(ERI_EINVAL, "shell " + std::to_string(s) + ": non-positive or non-finite exponent/coefficient");
      maxexp[s] = std::max(maxexp[s], a);
    }
    for (int d = 0; d < 3; ++d)
      if (!std::isfinite(basis->centers[3 * S.center + d])) return fail(ERI_EINVAL, "non-finite centre");
  }
  for (int64_t q = 0; q < 4 * nq; ++q)
    if (quartets[q] < 0 || quartets[q] >= nshell) return fail(ERI_EINVAL, "quartet index out of range");
  int rc = nq > 0 ? ensure_library() : ERI_OK;
  if (rc) return rc;
  Library& L = lib();

  auto plan = std::make_unique<eri_plan_s>();
  plan->nq = nq;
  plan->offsets.resize(nq + 1);
  plan->offsets[0] = 0;
  for (int64_t q = 0; q < nq; ++q) {
    int64_t sz = 1;
    for (int k = 0; k < 4; ++k) sz *= nfun(shells[quartets[4 * q + k]].l, cart);
    plan->offsets[q + 1] = plan->offsets[q] + sz;
  }
  if (nq == 0) {
    *plan_out = plan.release();
    return ERI_OK;
  }
  // ---- orientation and class of every quartet
  // Pair orientation.  Default: each primitive pair recurs on its tighter
  // primitive's centre (a contracted pair splits into at most two oriented
  // partial pairs), which keeps FP64 HRR cancellation bounded; options: the
  // whole pair on the shell with the largest exponent, or on the higher l.
  PairBuilder pb{shells, basis, &maxexp, opts.orientation, FlatMap(), {}, {}, 0};
  std::vector<DevPairIn>& pin = pb.pin;
  // molecule plans: alias records of chunked pairs, after the molecule's pairs
  std::vector<EriPairRec> mol_alias;
  // Chunks: a shell quartet of the team-cooperative tier evaluates its
  // primitive quartets one after another, so a deep contraction is cut into
  // chunks of about kCoopChunk primitive quartets (sub-ranges of the bra
  // pair's primitive pairs) that different teams run concurrently.
  const int kCoopChunk = 32;
  const bool default_opts = opts.axis_rule == 0 && opts.schedule == 0 && opts.sph_mode == 0;
  // Tier of a class at a precision: the caller's forced tier; FP32 forms on
  // the compiled register kernel, else the cooperative program; otherwise the
  // autotuner's choice when it is feasible, else the static rule (register,
  // cooperative, shared, global).  0 when no tier can hold the class (the
  // bucket loop reports why).  Chunking of deep contractions asks the same
  // question, so only buckets that run on the cooperative tier -- the one
  // that reduces chunks into their blocks -- are ever chunked.
  auto route_tier = [&](const int ls[4], int prec) -> int {
    const std::vector<int> pkey = {ls[0], ls[1], ls[2], ls[3], opts.axis_rule, opts.schedule, opts.sph_mode};
    auto pit = L.progs.find(pkey);
    const ClassProg* prog = pit == L.progs.end() ? nullptr : pit->second.get();
    const bool cp = L.coops.find(pkey) != L.coops.end();
    const auto& regmap = prec ? L.reg_f32 : L.reg;
    const bool regfn = default_opts && regmap.find({ls[0], ls[1], ls[2], ls[3]}) != regmap.end();
    const size_t smem_need = prog ? (size_t)prog->nslot * 128 * sizeof(double) : 0;
    // persistent plans: the compiled register-tier kernels keep their
    // classes (launches of their own, before the persistent launch); every
    // other class goes on the work list (tier 4 forces all of them there)
    if (persistent) return (opts.tier == 0 && regfn) ? TIER_REG : TIER_COOP;
    if (opts.tier != 0) return opts.tier;
    if (prec) return regfn ? TIER_REG : TIER_COOP;
    const int pt = preferred_tier(ls);
    const bool ok = (pt == TIER_REG && regfn) || (pt == TIER_COOP && cp) ||
                    (pt == TIER_SHARED && prog && smem_need <= L.smem_optin) || (pt == TIER_GLOBAL && prog);
    if (ok) return pt;
    return regfn ? TIER_REG : cp ? TIER_COOP : (prog && smem_need <= L.smem_optin ? TIER_SHARED : TIER_GLOBAL);
  };
  // class code ((la * 5 + lb) * 5 + lc) * 5 + ld, x2 for the precision;
  // per-code answers cached
  std::vector<int8_t> coop_of(2 * 625, -1);
  auto is_coop = [&](int la, int lb, int lc, int ld, int prec) {
    int8_t& c = coop_of[2 * (((la * 5 + lb) * 5 + lc) * 5 + ld) + prec];
    if (c < 0) {
      const int ls[4] = {la, lb, lc, ld};
      const std::vector<int> key = {la, lb, lc, ld, opts.axis_rule, opts.schedule, opts.sph_mode};
      c = (route_tier(ls, prec) == TIER_COOP && L.coops.find(key) != L.coops.end()) ? 1 : 0;
    }
    return c == 1;
  };
  FlatMap alias_id;
  auto get_alias = [&](int parent, int start, int count) {
    const uint64_t key = ((uint64_t)(uint32_t)parent << 32) | ((uint64_t)(uint32_t)start << 16) | (uint32_t)count;
    const int32_t found = alias_id.find(key);
    if (found >= 0) return (int)found;
    if (mol) {
      // a record pointing into the molecule's primitive pairs (its A - B as
      // the pair set-up kernel computes it)
      const DevPairIn& pd = mol->pb.pin[parent];
      const double* A = basis->centers + 3 * shells[pd.a].center;
      const double* Bc = basis->centers + 3 * shells[pd.b].center;
      EriPairRec r;
      r.prim_off = pd.prim_off + start;
      r.nprim = count;
      for (int d = 0; d < 3; ++d) r.AB[d] = A[d] - Bc[d];
      const int id = mol->npair + (int)mol_alias.size();
      mol_alias.push_back(r);
      alias_id.get_or_insert(key, [&] { return (int32_t)id; });
      return id;
    }
    DevPairIn d = pin[parent];
    d.prim_off += start;
    d.list_off = -2;
    d.nlist = count;
    const int id = (int)pin.size();
    pin.push_back(d);
    alias_id.get_or_insert(key, [&] { return (int32_t)id; });
    return id;
  };
  bool any_reduce = false;
  FlatMap split_id;
  std::vector<SplitRes> split_res;
  auto split = [&](int s0, int s1, PairPart* out) {
    if (s0 < s1) std::swap(s0, s1);
    const SplitRes* r;
    if (mol) {
      r = &mol->splits[(int64_t)s0 * (s0 + 1) / 2 + s1];
    } else {
      const uint64_t key = ((uint64_t)(uint32_t)s0 << 32) | (uint32_t)s1;
      const int32_t k = split_id.get_or_insert(key, [&] {
        SplitRes x;
        x.n = pb.split(s0, s1, x.part);
        split_res.push_back(x);
        return (int32_t)split_res.size() - 1;
      });
      r = &split_res[k];
    }
    out[0] = r->part[0];
    out[1] = r->part[1];
    return r->n;
  };
  struct QInfo {
    int cls;    // class key index
    int round;  // part number within its quartet: 0 writes the block, later parts add
    int kb, kk;
    int prec;   // 1: FP32 recurrences
    int32_t uq; // the caller's quartet
    EriQuartetRec rec;
  };
  // fused digestion (persistent digest plans): parts of every quartet
  const bool fuse = persistent && opts.digest == 1;
  // Parts of one quartet: in one launch round, reducing into the zeroed
  // block (the default; measured: the 60-atom water cluster runs 154
  // launches instead of 380 in the same 257 ms, the serving benchmark's
  // capacity rises from 183 to 264 requests/s), or one round per part
  // adding in order (opts.ordered).
  const bool one_round = opts.ordered == 0;
  std::vector<int32_t> nparts_q(fuse ? nq : 0, 0);
  // reduced precision is offered for the default generator options, where
  // every class has an FP32 form (register or team-cooperative tier)
  const bool mixed = qbound != nullptr && opts.axis_rule == 0 && opts.schedule == 0 && opts.sph_mode == 0 &&
                     (opts.tier == 0 || opts.tier == TIER_REG || opts.tier == TIER_COOP);
  std::vector<QInfo> qi;
  qi.reserve(nq + nq / 2);
  std::vector<int> cls_index(625, -1);  // class code -> class key index
  std::vector<std::vector<int>> cls_keys;
  for (int64_t q = 0; q < nq; ++q) {
    const int32_t* s = quartets + 4 * q;
    if (mol && q + 16 < nq) {
      // the molecule's split table holds every shell pair, and a request's
      // quartets index it at random: fetch quartet q + 16's entries early
      const int32_t* t = s + 64;
      const int64_t h0 = std::max(t[0], t[1]), l0 = std::min(t[0], t[1]);
      const int64_t h1 = std::max(t[2], t[3]), l1 = std::min(t[2], t[3]);
      __builtin_prefetch(&mol->splits[h0 * (h0 + 1) / 2 + l0]);
      __builtin_prefetch(&mol->splits[h1 * (h1 + 1) / 2 + l1]);
    }
    const int prec = mixed && qbound[q] < fp32_below ? 1 : 0;
    int n[4];
    for (int k = 0; k < 4; ++k) n[k] = nfun(shells[s[k]].l, cart);
    const int ustride[4] = {n[1] * n[2] * n[3], n[2] * n[3], n[3], 1};
    PairPart bp[2], kp[2];
    const int nb = split(s[0], s[1], bp), nk = split(s[2], s[3], kp);
    int round = 0;
    for (int ib = 0; ib < nb; ++ib)
      for (int ik = 0; ik < nk; ++ik, ++round) {
        PairPart B = bp[ib], K = kp[ik];
        // pos[k] = user position of canonical index k
        int pos[4] = {B.center == s[0] ? 0 : 1, B.center == s[0] ? 1 : 0, K.center == s[2] ? 2 : 3,
                      K.center == s[2] ? 3 : 2};
        if (s[0] == s[1]) pos[0] = 0, pos[1] = 1;
        if (s[2] == s[3]) pos[2] = 2, pos[3] = 3;
        int lb0 = shells[B.center].l, lb1 = shells[B.other].l, lk0 = shells[K.center].l, lk1 = shells[K.other].l;
        // bra-ket exchange so that the bra pair rank is not below the ket's
        if (lb0 * 5 + lb1 < lk0 * 5 + lk1) {
          std::swap(B, K);
          std::swap(pos[0], pos[2]);
          std::swap(pos[1], pos[3]);
          std::swap(lb0, lk0);
          std::swap(lb1, lk1);
        }
        int& cidx = cls_index[((lb0 * 5 + lb1) * 5 + lk0) * 5 + lk1];
        if (cidx < 0) {
          cidx = (int)cls_keys.size();
          cls_keys.push_back({lb0, lb1, lk0, lk1});
        }
        int cb = B.nprim, nchunk = 1;
        if ((int64_t)B.nprim * K.nprim > kCoopChunk && is_coop(lb0, lb1, lk0, lk1, prec)) {
          cb = std::max(1, kCoopChunk / K.nprim);
          nchunk = (B.nprim + cb - 1) / cb;
        }
        for (int c = 0; c < nchunk; ++c) {
          const int start = c * cb, cnt = std::min(cb, B.nprim - start);
          QInfo x;
          const int bpair = nchunk > 1 ? get_alias(B.pair, start, cnt) : B.pair;
          if (one_round) {
            // every part of a quartet with several reduces into its zeroed
            // block, in any order
            x.rec.bra = bpair | ((nb * nk > 1 || nchunk > 1) ? 0x40000000 : 0);
          } else {
            x.rec.bra = bpair | (round > 0 ? (int32_t)0x80000000 : 0) | (nchunk > 1 ? 0x40000000 : 0);
          }
          x.rec.ket = K.pair;
          x.rec.out_off = plan->offsets[q];
          for (int k = 0; k < 4; ++k) x.rec.st[k] = ustride[pos[k]];
          x.cls = cidx;
          x.round = one_round ? 0 : round;
          x.kb = cnt;
          x.kk = K.nprim;
          x.prec = prec;
          x.uq = (int32_t)q;
          // fused digestion counts the parts the persistent launch runs; a
          // quartet whose every part is register-tier is digested after it
          if (fuse && is_coop(lb0, lb1, lk0, lk1, prec)) ++nparts_q[q];
          qi.push_back(x);
        }
        if (nchunk > 1 || (one_round && nb * nk > 1)) any_reduce = true;
      }
  }
  const int64_t nparts = (int64_t)qi.size();
  plan->zero_out = any_reduce;
  if (pb.pprim > ((int64_t)1 << 31) - 1) return fail(ERI_EINVAL, "too many primitive pairs");
  // ---- buckets: by part round (a block is written before it is added to),
  // then class (heaviest first), precision, then contraction signature
  // (K4 descending, then bra depth descending).  One counting sort over a
  // dense key; equal keys keep their input order.
  std::vector<int> cls_rank(cls_keys.size());
  {
    std::vector<int> idx(cls_keys.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) {
      int sa = 0, sb = 0;
      for (int k = 0; k < 4; ++k) {
        sa += cls_keys[a][k];
        sb += cls_keys[b][k];
      }
      return sa != sb ? sa > sb : cls_keys[a] > cls_keys[b];
    });
    for (size_t r = 0; r < idx.size(); ++r) cls_rank[idx[r]] = (int)r;
  }
  const int64_t ncls = (int64_t)cls_keys.size();
  auto gid = [&](const QInfo& x) { return ((int64_t)x.round * ncls + cls_rank[x.cls]) * 2 + x.prec; };
  struct PartKey {
    int32_t cls, round, prec, kb, kk;
  };
  std::vector<PartKey> pk(nparts);
  std::vector<EriQuartetRec> recs(nparts);
  // record -> quartet: for the fused epilogue, and for the digestion lists
  // (ordered by the launch that evaluates a quartet's last part)
  std::vector<int32_t> rec_q(opts.digest == 1 ? nparts : 0);
  {
    // dense ids: used (round, class, precision) groups and (K4, kb) signatures
    std::vector<int32_t> gdense(4 * ncls * 2, -1);
    FlatMap sig_id;
    std::vector<std::pair<int64_t, int32_t>> sigs;  // (K4, kb)
    std::vector<uint32_t> key(nparts);
    // signatures of up to 64 x 64 primitive pairs (nearly all) by direct
    // lookup, the rest through the hash map
    constexpr int kSmallSig = 64;
    std::vector<int32_t> sig_small(kSmallSig * kSmallSig, -1);
    for (int64_t q = 0; q < nparts; ++q) {
      const QInfo& x = qi[q];
      gdense[gid(x)] = 0;
      auto make = [&] {
        sigs.push_back({(int64_t)x.kb * x.kk, x.kb});
        return (int32_t)sigs.size() - 1;
      };
      if (x.kb <= kSmallSig && x.kk <= kSmallSig) {
        int32_t& id = sig_small[(x.kb - 1) * kSmallSig + x.kk - 1];
        if (id < 0) id = make();
        key[q] = (uint32_t)id;
      } else {
        const uint64_t sk = ((uint64_t)(uint32_t)x.kb << 32) | (uint32_t)x.kk;
        key[q] = (uint32_t)sig_id.get_or_insert(sk, make);
      }
    }
    int32_t ng = 0;
    for (int32_t& g : gdense)
      if (g == 0) g = ng++;
    std::vector<int32_t> sig_rank(sigs.size());
    {
      std::vector<int32_t> idx(sigs.size());
      for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int32_t)i;
      std::sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return sigs[a] > sigs[b]; });
      for (size_t r = 0; r < idx.size(); ++r) sig_rank[idx[r]] = (int32_t)r;
    }
    const int64_t ns = (int64_t)sigs.size(), nkey = (int64_t)ng * ns;
    if (nkey > ((int64_t)1 << 27)) return fail(ERI_EUNSUPPORTED, "too many distinct contraction signatures");
    std::vector<int64_t> start(nkey + 1, 0);
    for (int64_t q = 0; q < nparts; ++q) {
      key[q] = (uint32_t)(gdense[gid(qi[q])] * ns + sig_rank[key[q]]);
      ++start[key[q] + 1];
    }
    for (int64_t k = 0; k < nkey; ++k) start[k + 1] += start[k];
    for (int64_t q = 0; q < nparts; ++q) {
      const QInfo& x = qi[q];
      const int64_t p = start[key[q]]++;
      recs[p] = x.rec;
      if (opts.digest == 1) rec_q[p] = x.uq;
      pk[p] = {x.cls, x.round, x.prec, x.kb, x.kk};
    }
  }
  std::vector<QInfo>().swap(qi);  // release the unsorted parts
  // ---- launches: one per (class, group size); G lanes share a quartet and
  // split its K4 primitive quartets: about three primitive quartets per lane,
  // but no more lanes than needed to give the launch ~16 warps per SM (every
  // extra lane costs a share of the accumulator reduction).  run_len[i] =
  // the number of parts with part i's (round, class, precision, K4): a run of
  // the sorted order.
  auto same_group = [](const PartKey& a, const PartKey& b) {
    return a.cls == b.cls && a.round == b.round && a.prec == b.prec;
  };
  std::vector<int64_t> run_len(nparts);
  for (int64_t i = 0; i < nparts;) {
    const int64_t k4 = (int64_t)pk[i].kb * pk[i].kk;
    int64_t j = i + 1;
    while (j < nparts && same_group(pk[j], pk[i]) && (int64_t)pk[j].kb * pk[j].kk == k4) ++j;
    for (int64_t t = i; t < j; ++t) run_len[t] = j - i;
    i = j;
  }
  const int64_t lanes_target = (int64_t)L.nsm * 512;
  auto group_at = [&](int64_t i) {
    const int64_t k4 = (int64_t)pk[i].kb * pk[i].kk;
    int64_t want = std::min<int64_t>(32, std::max<int64_t>(1, (k4 + 2) / 3));
    want = std::min<int64_t>(want, std::max<int64_t>(1, lanes_target / std::max<int64_t>(1, run_len[i])));
    int g = 1;
    while (g * 2 <= want) g *= 2;
    return g;
  };
  size_t max_scratch_slots = 0;
  int max_grid_global = 0;
  size_t max_coop_vals = 0, max_coop_h = 0;
  for (int64_t i = 0; i < nparts;) {
    const int c = pk[i].cls;
    const int round = pk[i].round;
    const int prec = pk[i].prec;
    Bucket b;
    b.fp32 = prec;
    for (int k = 0; k < 4; ++k) b.ls[k] = cls_keys[c][k];
    std::vector<int> pkey = {b.ls[0], b.ls[1], b.ls[2], b.ls[3], opts.axis_rule, opts.schedule, opts.sph_mode};
    auto pit = L.progs.find(pkey);
    ClassProg* prog = pit == L.progs.end() ? nullptr : pit->second.get();
    auto cit = L.coops.find(pkey);
    CoopProg* cp = cit == L.coops.end() ? nullptr : cit->second.get();
    const auto& regmap = prec ? L.reg_f32 : L.reg;
    auto rit = regmap.find({b.ls[0], b.ls[1], b.ls[2], b.ls[3]});
    const void* regfn = (rit != regmap.end() && default_opts) ? rit->second : nullptr;
    const size_t smem_need = prog ? (size_t)prog->nslot * 128 * sizeof(double) : 0;
    const int tier = route_tier(b.ls, prec);
    if (tier == TIER_REG && !regfn)
      return fail(ERI_EUNSUPPORTED, "no register-tier kernel for this class/options");
    if (tier == TIER_COOP && !cp)
      return fail(ERI_EUNSUPPORTED, "no team-cooperative program for this class/options");
    if ((tier == TIER_SHARED || tier == TIER_GLOBAL) && !prog)
      return fail(ERI_EUNSUPPORTED, "no program for this class/options (build the variant)");
    if (tier == TIER_SHARED && smem_need > L.smem_optin)
      return fail(ERI_EUNSUPPORTED, "class does not fit the shared-memory tier");
    // one launch per class for the cooperative tier (a team walks all the
    // primitive quartets of its shell quartet); otherwise one per group size
    const int g = tier == TIER_COOP ? 1 : group_at(i);
    // K4 of the bucket's first (deepest) part; cooperative buckets split at
    // the shallow-contraction boundary
    // (deep > kShallowK4 >= shallow > 1 = single primitive quartet)
    const int64_t k4_first = (int64_t)pk[i].kb * pk[i].kk;
    auto coop_cat = [](int64_t k4) { return k4 == 1 ? 2 : (k4 <= kShallowK4 ? 1 : 0); };
    const bool shallow = tier == TIER_COOP && k4_first <= kShallowK4;
    int64_t j = i;
    double kprim = 0;
    while (j < nparts && pk[j].cls == c && pk[j].round == round && pk[j].prec == prec &&
           (tier == TIER_COOP ? coop_cat((int64_t)pk[j].kb * pk[j].kk) == coop_cat(k4_first)
                              : group_at(j) == g)) {
      kprim += (double)pk[j].kb * pk[j].kk;
      ++j;
    }
    b.first = i;
    b.count = j - i;
    b.group = g;
    b.tier = tier;
    b.reg_fn = regfn;
    b.prog = prog;
    const int64_t blocks = (b.count * g + 127) / 128;
    if (tier == TIER_REG) {
      b.grid = (int)blocks;
    } else if (tier == TIER_SHARED) {
      b.smem = smem_need;
      int per_sm = (int)std::max<size_t>(1, std::min<size_t>(4, (L.smem_optin + 1024) / (smem_need + 1024)));
      b.grid = (int)std::min<int64_t>(blocks, (int64_t)L.nsm * per_sm);
    } else if (tier == TIER_GLOBAL) {
      int per_sm = prog->nslot <= 4096 ? 4 : 2;
      b.grid = (int)std::min<int64_t>(blocks, (int64_t)L.nsm * per_sm);
      max_scratch_slots = std::max(max_scratch_slots, (size_t)prog->nslot);
      max_grid_global = std::max(max_grid_global, b.grid);
    } else {
      // team-cooperative: value slots (and H when it fits) in shared memory.
      // Pick the block shape (teams per block) and the H placement that keep
      // the most warps resident per SM, up to 16.
      if (shallow) {
        auto sit = L.coops_shallow.find(pkey);
        if (sit != L.coops_shallow.end()) cp = sit->second.get();
      }
      // the autotuner's shape for this class and kind of contraction
      const int kind = coop_cat(k4_first);
      int pshape = -1, pvotes = 0;
      const std::vector<CoopProg*> shapes = class_shapes(L, pkey);
      if (default_opts && preferred_shape(b.ls, kind, &pshape, &pvotes) && pshape >= 0 &&
          pshape < (int)shapes.size())
        cp = shapes[pshape];
      b.kind = kind;
      b.shape = (int)(std::find(shapes.begin(), shapes.end(), cp) - shapes.begin());
      // warp votes around the optional FP64 terms: on request, else the
      // class table's preference (autotuner), else the static rule, measured
      // on the sweep classes with K per shell from {1, 3, 6}: votes pay for
      // teams of 128 lanes or more ((ff|ff) 0.610 -> 0.690 of the FP64 rate,
      // (gg|gg) 0.620 -> 0.632) and cost 64-lane teams ((dd|dd) 0.602 -> 0.582);
      // single-primitive parts of 512-lane teams run better predicated
      // (autotuner, (gg|gg) at K = 1: 0.485 -> 0.513)
      {
        const int pv = pvotes ? pvotes : preferred_votes(b.ls);
        const int stat = cp->T >= 512 && k4_first == 1 ? 1 : cp->T >= 128 ? 2 : 1;
        const int want_v = opts.votes ? opts.votes : pv ? pv : stat;
        b.vote = want_v == 2 ? 1 : 0;
      }
      b.coop = cp;
      // single-primitive parts: a team computes the rows of kShallowK4
      // consecutive quartets at once
      b.single = k4_first == 1 ? 1 : 0;
      b.batch = b.single ? kShallowK4
                         : (int)std::min<int64_t>(eri_coop_max_batch(), std::max<int64_t>(1, k4_first));
      const size_t smem_sm = L.smem_per_sm, reserve = 1024;
      int best_warps = -1;
      const size_t rows = eri_coop_row_elems() * (size_t)b.batch;
      const size_t elem = prec ? sizeof(float) : sizeof(double);
      for (int h_in = 1; h_in >= 0; --h_in) {
        for (int tpb = std::max(1, 128 / cp->T); tpb >= 1; tpb /= 2) {
          // every value slot lives in shared memory; H too when it fits
          const size_t per_team = rows + cp->nslot + (h_in ? (size_t)cp->nh : 0);
          if (per_team * tpb * elem > L.smem_optin) continue;
          const size_t bsm = (per_team * tpb * elem + 15) / 16 * 16;
          // registers: the 4-nodes-per-lane kernels hold ~230 registers, so at
          // most 256 of their threads per SM; the others at most 512
          const size_t max_threads = cp->ilp == 4 ? 256 : 512;
          const int bps = (int)std::min<size_t>(max_threads / (tpb * cp->T), std::max<size_t>(1, smem_sm / (bsm + reserve)));
          if (bps < 1) continue;
          const int warps = bps * tpb * cp->T / 32;
          // prefer H in shared memory at equal residency
          if (warps > best_warps) {
            best_warps = warps;
            b.h_in_smem = h_in;
            b.smem_slots = cp->nslot;
            b.smem = bsm;
            b.block = tpb * cp->T;
            b.grid = bps;  // blocks per SM for now
          }
        }
      }
      if (best_warps < 0)
        return fail(ERI_EUNSUPPORTED, "class does not fit the team-cooperative tier's shared memory");
      const int tpb = b.block / cp->T;
      b.grid = (int)std::min<int64_t>((b.count + tpb - 1) / tpb, (int64_t)L.nsm * b.grid);
      b.nteams = b.grid * tpb;
      max_coop_vals = std::max(max_coop_vals, (size_t)b.nteams * (cp->nslot - b.smem_slots));
      if (!b.h_in_smem) max_coop_h = std::max(max_coop_h, (size_t)b.nteams * cp->nh);
      if ((rc = upload_coop(cp))) return rc;
    }
    if (prog) {
      if ((tier == TIER_SHARED || tier == TIER_GLOBAL) && (rc = upload_prog(prog))) return rc;
      b.flops = kprim * prog->flops_prim + (double)b.count * prog->flops_p2;
      if (prec) {
        plan->flops32 += b.flops;
        plan->nparts32 += b.count;
      } else {
        plan->flops += b.flops;
      }
    }
    plan->nprimq += kprim;
    b.round = round;
    b.shared_scratch = tier == TIER_GLOBAL || (tier == TIER_COOP && (!b.h_in_smem || b.smem_slots < cp->nslot));
    plan->buckets.push_back(b);
    i = j;
  }
  // ---- persistent plans: the cooperative buckets become work items of one
  // launch per (precision, vote form); a block of 512 threads per SM takes
  // items from a counter.  Per bucket: the team shape of its program, the
  // teams per block that fit the launch's shared memory (H in shared memory
  // when that keeps as many teams), and items of `teams` x r quartets, r
  // chosen for about eight items per SM per bucket.  Items go heaviest
  // bucket first so that the dynamic queue ends evenly.
  if (persistent) {
    std::vector<Bucket> groups;
    std::vector<EriWorkItem> items;
    std::vector<EriCoopProgDesc> progs;
    std::map<const CoopProg*, int> prog_id;
    const size_t smax = eri_coop_persist_smem_max(L.smem_optin);
    size_t smem_need = 0;
    int64_t gh_need = 0;
    for (int prec = 0; prec < 2; ++prec) {
      for (int vote = 0; vote < 2; ++vote) {
        std::vector<const Bucket*> bs;
        for (const Bucket& b : plan->buckets)
          if (b.tier == TIER_COOP && b.fp32 == prec && b.vote == vote) bs.push_back(&b);
        if (bs.empty()) continue;
        std::stable_sort(bs.begin(), bs.end(), [](const Bucket* x, const Bucket* y) {
          return x->flops / std::max<int64_t>(1, x->count) > y->flops / std::max<int64_t>(1, y->count);
        });
        Bucket g;
        g.tier = TIER_PERSIST;
        for (int k = 0; k < 4; ++k) g.ls[k] = -1;
        g.fp32 = prec;
        g.vote = vote;
        g.pgroup = (int)groups.size();
        g.item0 = (int)items.size();
        g.block = 512;
        g.grid = L.nsm;
        const size_t elem = prec ? sizeof(float) : sizeof(double);
        for (const Bucket* b : bs) {
          // the persistent kernel runs two nodes per lane (512 threads per
          // SM leave 128 registers a thread); a bucket whose shape takes
          // four falls back to the class's first shipped two-node shape
          const CoopProg* cp = b->coop;
          if (cp->ilp != 2) {
            const CoopProg* alt = nullptr;
            for (const CoopProg* c : class_shapes(L, {b->ls[0], b->ls[1], b->ls[2], b->ls[3], opts.axis_rule,
                                                      opts.schedule, opts.sph_mode}))
              if (c->ilp == 2 && c->T <= 512) {
                alt = c;
                break;
              }
            if (!alt) return fail(ERI_EUNSUPPORTED, "no two-node cooperative shape for the persistent launch");
            if ((rc = upload_coop(const_cast<CoopProg*>(alt)))) return rc;
            cp = alt;
          }
          auto pit = prog_id.find(cp);
          if (pit == prog_id.end()) {
            EriCoopProgDesc d;
            d.ph1 = cp->d_ph1;
            d.steps1 = cp->d_steps1;
            d.ph2 = cp->d_ph2;
            d.steps2 = cp->d_steps2;
            d.nw1 = cp->nw1;
            d.nw2 = cp->nw2;
            d.nh = cp->nh;
            d.nslot = cp->nslot;
            d.L = cp->L;
            d.pad = 0;
            pit = prog_id.emplace(cp, (int)progs.size()).first;
            progs.push_back(d);
          }
          const size_t rows = eri_coop_row_elems() * (size_t)b->batch;
          int best = 0, hsm = 0;
          for (int h_in = 1; h_in >= 0; --h_in) {
            const size_t per_team = (rows + cp->nslot + (h_in ? (size_t)cp->nh : 0)) * elem;
            const int t = (int)std::min<size_t>(512 / cp->T, smax / per_team);
            if (t > best) best = t, hsm = h_in;
          }
          if (best < 1) return fail(ERI_EUNSUPPORTED, "class does not fit the persistent launch's shared memory");
          const size_t per_team = rows + cp->nslot + (hsm ? (size_t)cp->nh : 0);
          smem_need = std::max(smem_need, (per_team * best * elem + 15) / 16 * 16);
          if (!hsm) gh_need = std::max<int64_t>(gh_need, (int64_t)best * cp->nh);
          const int64_t r = std::max<int64_t>(1, (b->count + (int64_t)best * 8 * L.nsm - 1) /
                                                     ((int64_t)best * 8 * L.nsm));
          const int64_t per_item = r * best;
          for (int64_t f = 0; f < b->count; f += per_item) {
            EriWorkItem w;
            w.prog = pit->second;
            w.first = (int32_t)(b->first + f);
            w.count = (int32_t)std::min<int64_t>(per_item, b->count - f);
            w.T = (int16_t)cp->T;
            w.teams = (int16_t)best;
            w.hsm = (int8_t)hsm;
            w.vote = (int8_t)vote;
            w.single = (int8_t)b->single;
            w.pad = 0;
            w.batch = b->batch;
            items.push_back(w);
          }
          g.count += b->count;
          g.flops += b->flops;
        }
        g.nitems = (int)items.size() - g.item0;
        groups.push_back(g);
      }
    }
    if (items.size() > (size_t)INT32_MAX) return fail(ERI_EUNSUPPORTED, "too many work items");
    for (Bucket& g : groups) g.smem = smem_need;
    // the register-tier buckets first, then the persistent launches
    std::vector<Bucket> all;
    for (const Bucket& b : plan->buckets)
      if (b.tier != TIER_COOP) all.push_back(b);
    all.insert(all.end(), groups.begin(), groups.end());
    plan->buckets = all;
    plan->persistent = true;
    plan->persist_h_per_block = gh_need;
    if ((rc = plan->items.upload(items, "work items")) || (rc = plan->progs.upload(progs, "program table")) ||
        (rc = plan->counters.alloc(std::max<size_t>(1, groups.size()), "item counters")) ||
        (rc = plan->persist_h.alloc((size_t)gh_need * L.nsm, "persistent accumulators")))
      return rc;
  }
  // ---- concurrency: the launches of one part round write distinct blocks,
  // so they may overlap on several streams (fork/join per round); launches
  // on the plan's global scratch stay on the caller's stream.  Greedy
  // assignment, heaviest class first, by estimated cost (flops plus a fixed
  // per-launch share).
  {
    std::set<std::vector<int>> classes;
    for (const Bucket& b : plan->buckets) classes.insert({b.ls[0], b.ls[1], b.ls[2], b.ls[3]});
    // a persistent plan's launches each fill the GPU: one stream
    const int want = persistent ? 1 : opts.streams > 0 ? opts.streams : (classes.size() > 1 ? 4 : 1);
    int used = 1;
    for (size_t i = 0; i < plan->buckets.size();) {
      size_t j = i;
      while (j < plan->buckets.size() && plan->buckets[j].round == plan->buckets[i].round) ++j;
      std::vector<double> load(want, 0.0);
      for (size_t k = i; k < j; ++k) {
        Bucket& b = plan->buckets[k];
        int lane = 0;
        if (!b.shared_scratch)
          for (int l = 1; l < want; ++l)
            if (load[l] < load[lane]) lane = l;
        b.lane = lane;
        load[lane] += b.flops + 2e7;
        used = std::max(used, lane + 1);
      }
      i = j;
    }
    plan->nlanes = used;
    if (used > 1) {
      CUDA_OR(cudaEventCreateWithFlags(&plan->fork_ev, cudaEventDisableTiming), "cudaEventCreate");
      for (int l = 1; l < used; ++l) {
        cudaStream_t st;
        cudaEvent_t ev;
        CUDA_OR(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "cudaStreamCreate");
        plan->lanes.push_back(st);
        CUDA_OR(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "cudaEventCreate");
        plan->join_ev.push_back(ev);
      }
    }
  }
  if ((rc = plan->coop_vals.alloc(max_coop_vals, "cooperative spill")) ||
      (rc = plan->coop_h.alloc(max_coop_h, "cooperative accumulators")))
    return rc;
  // ---- device data
  std::vector<DevShell> dsh;
  std::vector<double> ex, co;
  if (mol) {
    // the molecule's shells and primitive pairs stay where they are; the plan
    // holds a copy of its pair records, followed by this plan's aliases
    const size_t npr = (size_t)mol->npair + mol_alias.size();
    if ((rc = plan->pairs.alloc(npr, "pairs")) || (rc = plan->quartets.upload(recs, "quartet records"))) return rc;
    if (plan->pairs.async) {
      CUDA_OR(cudaMemcpyAsync(plan->pairs.p, mol->pairs_d.p, (size_t)mol->npair * sizeof(EriPairRec),
                              cudaMemcpyDeviceToDevice, plan->pairs.st), "copy molecule pairs");
      if (!mol_alias.empty())
        CUDA_OR(cudaMemcpyAsync(plan->pairs.p + mol->npair, mol_alias.data(), mol_alias.size() * sizeof(EriPairRec),
                                cudaMemcpyHostToDevice, plan->pairs.st), "upload aliases");
    } else {
      CUDA_OR(cudaMemcpy(plan->pairs.p, mol->pairs_d.p, (size_t)mol->npair * sizeof(EriPairRec),
                         cudaMemcpyDeviceToDevice), "copy molecule pairs");
      if (!mol_alias.empty())
        CUDA_OR(cudaMemcpy(plan->pairs.p + mol->npair, mol_alias.data(), mol_alias.size() * sizeof(EriPairRec),
                           cudaMemcpyHostToDevice), "upload aliases");
    }
    plan->mol = mol;
    plan->npair = 0;  // nothing for the pair set-up kernel
    plan->npprim = mol->pb.pprim;
  } else {
    dsh.resize(nshell);
    for (int s = 0; s < nshell; ++s) {
      for (int d = 0; d < 3; ++d) dsh[s].ctr[d] = basis->centers[3 * shells[s].center + d];
      dsh[s].l = shells[s].l;
      dsh[s].nprim = shells[s].nprim;
      dsh[s].prim = shells[s].prim_offset;
      dsh[s].pad = 0;
    }
    ex.assign(basis->exponents, basis->exponents + basis->nprim_total);
    co.assign(basis->coefs, basis->coefs + basis->nprim_total);
    if ((rc = plan->shells.upload(dsh, "shells")) || (rc = plan->exps.upload(ex, "exponents")) ||
        (rc = plan->coefs.upload(co, "coefficients")) || (rc = plan->pin.upload(pin, "pair list")) ||
        (rc = plan->plist.upload(pb.plist, "primitive-pair lists")) ||
        (rc = plan->pairs.alloc(pin.size(), "pairs")) || (rc = plan->pprims.alloc(pb.pprim, "primitive pairs")) ||
        (plan->nparts32 > 0 && (rc = plan->pprims_f.alloc(pb.pprim, "primitive pairs (FP32)"))) ||
        (rc = plan->quartets.upload(recs, "quartet records")))
      return rc;
    plan->npair = (int)pin.size();
    plan->npprim = pb.pprim;
  }
  {
    // a plan whose every quartet is (ab|ab) can also produce Schwarz bounds
    bool diag = true;
    for (int64_t q = 0; q < nq && diag; ++q) {
      const int32_t* s4 = quartets + 4 * q;
      diag = s4[0] == s4[2] && s4[1] == s4[3];
    }
    std::vector<int32_t> nab(diag ? nq : 0);
    for (int64_t q = 0; q < (int64_t)nab.size(); ++q) {
      const int32_t* s4 = quartets + 4 * q;
      nab[q] = nfun(shells[s4[0]].l, cart) * nfun(shells[s4[1]].l, cart);
    }
    if (diag || opts.digest) {
      // nq + 1 entries: block starts and the total
      if ((rc = plan->d_offsets.upload(plan->offsets, "offsets"))) return rc;
    }
    if (diag) {
      plan->nab = nab;
      if ((rc = plan->d_nab.upload(nab, "pair sizes"))) return rc;
    }
  }
  if (fuse) {
    if ((rc = plan->rec_q.upload(rec_q, "record quartets")) || (rc = plan->nparts_q.upload(nparts_q, "part counts")) ||
        (rc = plan->done_q.alloc((size_t)nq, "part counters")))
      return rc;
  }
  if (opts.digest) {
    std::vector<int32_t> uq(quartets, quartets + 4 * nq);
    std::vector<int32_t> bf(nshell + 1, 0);
    for (int s = 0; s < nshell; ++s) bf[s + 1] = bf[s] + nfun(shells[s].l, cart);
    std::vector<int64_t> small, large, rsmall, rlarge;
    // the lists hold the quartets grouped by the launch (bucket) that
    // evaluates their last part (the highest part round; quartets whose
    // parts all run in a persistent launch come last), bucket by bucket, in
    // increasing quartet order within a bucket: the 32 quartets of a warp of
    // the small-block kernel then mostly belong to one class, with blocks of
    // one size, and take the same loop bounds (in quartet order the warp's
    // classes mix: measured on the 60-atom water cluster, 54 ms in quartet
    // order against 36.5 ms grouped)
    const size_t nbk = plan->buckets.size();
    std::vector<int32_t> lastb(nq, (int32_t)nbk);
    for (size_t k = 0; k < nbk; ++k) {
      const Bucket& b = plan->buckets[k];
      if (b.tier == TIER_PERSIST) continue;
      for (int64_t r = b.first; r < b.first + b.count; ++r) lastb[rec_q[r]] = (int32_t)k;
    }
    std::vector<int64_t> start(nbk + 2, 0), order(nq);
    for (int64_t q = 0; q < nq; ++q) ++start[lastb[q] + 1];
    for (size_t k = 0; k <= nbk; ++k) start[k + 1] += start[k];
    for (int64_t q = 0; q < nq; ++q) order[start[lastb[q]]++] = q;
    std::vector<int32_t>().swap(lastb);
    for (const int64_t q : order) {
      const bool sm = plan->offsets[q + 1] - plan->offsets[q] <= kSmallBlock;
      (sm ? small : large).push_back(q);
      if (fuse && nparts_q[q] == 0) (sm ? rsmall : rlarge).push_back(q);
    }
    if ((rc = plan->d_uq.upload(uq, "quartet list")) || (rc = plan->d_shell_bf.upload(bf, "shell offsets")) ||
        (rc = plan->d_small.upload(small, "digest list")) || (rc = plan->d_large.upload(large, "digest list")) ||
        (rc = plan->d_rsmall.upload(rsmall, "digest list")) || (rc = plan->d_rlarge.upload(rlarge, "digest list")))
      return rc;
    plan->nbf = bf[nshell];
    plan->digest = true;
    // triangle scratch for the digestion (one reduction per mirrored pair of
    // J and K entries instead of two), when it is at most 1 GiB
    const size_t tri = 2 * (size_t)plan->nbf * (size_t)plan->nbf;
    if (tri > 0 && tri * sizeof(double) <= ((size_t)1 << 30) && (rc = plan->jk_tri.alloc(tri, "J/K triangles")))
      return rc;
  }
  plan->h2d_bytes = (double)(dsh.size() * sizeof(DevShell) + 2 * ex.size() * sizeof(double) +
                             (mol ? mol_alias.size() * sizeof(EriPairRec)
                                  : pin.size() * sizeof(DevPairIn) + pb.plist.size() * sizeof(uint32_t)) +
                             recs.size() * sizeof(EriQuartetRec));
  if (max_scratch_slots > 0) {
    plan->scratch_stride = (int64_t)max_grid_global * 128;
    if ((rc = plan->scratch.alloc((size_t)plan->scratch_stride * max_scratch_slots, "scratch"))) return rc;
  }
  *plan_out = plan.release();
  return ERI_OK;
}

extern "C" int eri_plan(const eri_shell* shells, int32_t nshell, const eri_basis* basis, const int32_t* quartets,
                        int64_t nq, const eri_opts* opts, eri_plan_t** plan_out) {
  return plan_impl(shells, nshell, basis, quartets, nq, nullptr, 0.0, opts, plan_out);
}

extern "C" int eri_plan_on_stream(const eri_shell* shells, int32_t nshell, const eri_basis* basis,
                                  const int32_t* quartets, int64_t nq, const double* qbound, double fp32_below,
                                  const eri_opts* opts, void* stream, eri_plan_t** plan_out) {
  if (!stream) return fail(ERI_EINVAL, "stream-ordered plans need a non-default stream");
  if (qbound)
    for (int64_t q = 0; q < nq; ++q)
      if (!(qbound[q] >= 0)) return fail(ERI_EINVAL, "negative or NaN Schwarz bound");
  if (qbound && (!(fp32_below >= 0) || !std::isfinite(fp32_below))) return fail(ERI_EINVAL, "bad FP32 threshold");
  int rc;
  {
    AllocStreamScope scope((cudaStream_t)stream, true);
    rc = plan_impl(shells, nshell, basis, quartets, nq, qbound, fp32_below, opts, plan_out);
  }
  if (rc == ERI_OK && *plan_out) {
    (*plan_out)->stream_ordered = true;
    (*plan_out)->alloc_stream = (cudaStream_t)stream;
  }
  return rc;
}

extern "C" int eri_mol_create(const eri_shell* shells, int32_t nshell, const eri_basis* basis,
                                const eri_opts* opts_in, eri_mol_t** out) {
  if (!out) return fail(ERI_EINVAL, "out is NULL");
  *out = nullptr;
  eri_opts opts;
  memset(&opts, 0, sizeof opts);
  if (opts_in) opts = *opts_in;
  if (opts.orientation < 0 || opts.orientation > 2) return fail(ERI_EINVAL, "option out of range");
  if (nshell < 1 || !shells || !basis || !basis->centers || !basis->exponents || !basis->coefs ||
      basis->ncenter < 0 || basis->nprim_total < 0)
    return fail(ERI_EINVAL, "NULL or empty basis");
  auto m = std::make_unique<eri_mol_s>();
  m->nshell = nshell;
  m->orientation = opts.orientation;
  m->shells.assign(shells, shells + nshell);
  m->maxexp.assign(nshell, 0.0);
  for (int s = 0; s < nshell; ++s) {
    const eri_shell& S = shells[s];
    if (S.l < 0) return fail(ERI_EINVAL, "shell " + std::to_string(s) + ": negative l");
    if (S.l > ERI_MAX_L) return fail(ERI_EUNSUPPORTED, "shell " + std::to_string(s) + ": l > 4");
    if (S.nprim < 1 || S.nprim > ERI_MAX_NPRIM) return fail(ERI_EINVAL, "shell " + std::to_string(s) + ": bad nprim");
    if (S.center < 0 || S.center >= basis->ncenter) return fail(ERI_EINVAL, "shell " + std::to_string(s) + ": bad centre");
    if (S.prim_offset < 0 || (int64_t)S.prim_offset + S.nprim > basis->nprim_total)
      return fail(ERI_EINVAL, "shell " + std::to_string(s) + ": primitives out of range");
    for (int k = 0; k < S.nprim; ++k) {
      const double a = basis->exponents[S.prim_offset + k], c = basis->coefs[S.prim_offset + k];
      if (!(a > 0) || !std::isfinite(a) || !std::isfinite(c))
        return fail(ERI_EINVAL, "shell " + std::to_string(s) + ": non-positive or non-finite exponent/coefficient");
      m->maxexp[s] = std::max(m->maxexp[s], a);
    }
    for (int d = 0; d < 3; ++d)
      if (!std::isfinite(basis->centers[3 * S.center + d])) return fail(ERI_EINVAL, "non-finite centre");
  }
  m->centers.assign(basis->centers, basis->centers + 3 * (size_t)basis->ncenter);
  m->exps.assign(basis->exponents, basis->exponents + basis->nprim_total);
  m->coefs.assign(basis->coefs, basis->coefs + basis->nprim_total);
  m->view = eri_basis{m->centers.data(), basis->ncenter, m->exps.data(), m->coefs.data(), basis->nprim_total};
  int rc = ensure_library();
  if (rc) return rc;
  m->pb.shells = m->shells.data();
  m->pb.basis = &m->view;
  m->pb.maxexp = &m->maxexp;
  m->pb.orientation = opts.orientation;
  const int64_t npairs = (int64_t)nshell * (nshell + 1) / 2;
  m->splits.resize(npairs);
  for (int a = 0; a < nshell; ++a)
    for (int b = 0; b <= a; ++b) {
      SplitRes& r = m->splits[(int64_t)a * (a + 1) / 2 + b];
      r.n = m->pb.split(a, b, r.part);
    }
  if (m->pb.pprim > ((int64_t)1 << 31) - 1) return fail(ERI_EINVAL, "too many primitive pairs");
  m->npair = (int)m->pb.pin.size();
  std::vector<DevShell> dsh(nshell);
  for (int s = 0; s < nshell; ++s) {
    for (int d = 0; d < 3; ++d) dsh[s].ctr[d] = m->centers[3 * shells[s].center + d];
    dsh[s].l = shells[s].l;
    dsh[s].nprim = shells[s].nprim;
    dsh[s].prim = shells[s].prim_offset;
    dsh[s].pad = 0;
  }
  if ((rc = m->shells_d.upload(dsh, "shells")) || (rc = m->exps_d.upload(m->exps, "exponents")) ||
      (rc = m->coefs_d.upload(m->coefs, "coefficients")) || (rc = m->pin_d.upload(m->pb.pin, "pair list")) ||
      (rc = m->plist_d.upload(m->pb.plist, "primitive-pair lists")) ||
      (rc = m->pairs_d.alloc(m->npair, "pairs")) || (rc = m->pprims_d.alloc(m->pb.pprim, "primitive pairs")) ||
      (rc = m->pprims_f.alloc(m->pb.pprim, "primitive pairs (FP32)")))
    return rc;
  const int threads = 128;
  eri_pair_setup_kernel<<<(m->npair + threads - 1) / threads, threads>>>(
      m->pin_d.p, m->npair, m->shells_d.p, m->exps_d.p, m->coefs_d.p, m->plist_d.p, m->pairs_d.p, m->pprims_d.p,
      m->pprims_f.p);
  CUDA_OR(cudaGetLastError(), "pair set-up launch");
  CUDA_OR(cudaDeviceSynchronize(), "pair set-up");
  *out = m.release();
  return ERI_OK;
}

extern "C" int eri_mol_destroy(eri_mol_t* mol) {
  if (!mol) return ERI_OK;
  cudaDeviceSynchronize();
  delete mol;
  return ERI_OK;
}

extern "C" int eri_plan_on_mol(const eri_mol_t* mol, const int32_t* quartets, int64_t nq, const double* qbound,
                                 double fp32_below, const eri_opts* opts, void* stream, eri_plan_t** plan_out) {
  if (!mol) return fail(ERI_EINVAL, "NULL molecule");
  if (qbound)
    for (int64_t q = 0; q < nq; ++q)
      if (!(qbound[q] >= 0)) return fail(ERI_EINVAL, "negative or NaN Schwarz bound");
  if (qbound && (!(fp32_below >= 0) || !std::isfinite(fp32_below))) return fail(ERI_EINVAL, "bad FP32 threshold");
  int rc;
  {
    AllocStreamScope scope((cudaStream_t)stream, stream != nullptr);
    rc = plan_impl(nullptr, 0, nullptr, quartets, nq, qbound, fp32_below, opts, plan_out, mol);
  }
  if (rc == ERI_OK && *plan_out && stream) {
    (*plan_out)->stream_ordered = true;
    (*plan_out)->alloc_stream = (cudaStream_t)stream;
  }
  return rc;
}

extern "C" int eri_plan_mixed(const eri_shell* shells, int32_t nshell, const eri_basis* basis,
                              const int32_t* quartets, int64_t nq, const double* qbound, double fp32_below,
                              const eri_opts* opts, eri_plan_t** plan_out) {
  if (nq > 0 && !qbound) return fail(ERI_EINVAL, "NULL bound array");
  if (!(fp32_below >= 0) || !std::isfinite(fp32_below)) return fail(ERI_EINVAL, "bad FP32 threshold");
  for (int64_t q = 0; q < nq; ++q)
    if (!(qbound[q] >= 0)) return fail(ERI_EINVAL, "negative or NaN Schwarz bound");
  return plan_impl(shells, nshell, basis, quartets, nq, qbound, fp32_below, opts, plan_out);
}

extern "C" int64_t eri_output_count(const eri_plan_t* plan) { return plan ? plan->offsets.back() : 0; }

extern "C" int eri_output_offsets(const eri_plan_t* plan, int64_t* offsets) {
  if (!plan || !offsets) return fail(ERI_EINVAL, "NULL argument");
  memcpy(offsets, plan->offsets.data(), plan->offsets.size() * sizeof(int64_t));
  return ERI_OK;
}

// Digestion fused into a persistent plan's launch (eri_compute_jk).
struct FuseIn {
  const double* D;
  double* J;
  double* K;
  int32_t nbf;
};

static int compute_impl(eri_plan_t* plan, double* out, void* stream_, const FuseIn* fz);

extern "C" int eri_compute(eri_plan_t* plan, double* out, void* stream_) {
  return compute_impl(plan, out, stream_, nullptr);
}

static int compute_impl(eri_plan_t* plan, double* out, void* stream_, const FuseIn* fz) {
  if (!plan) return fail(ERI_EINVAL, "NULL plan");
  if (plan->nq == 0) return ERI_OK;
  if (!out) return fail(ERI_EINVAL, "NULL output");
  if (((uintptr_t)out & 7) != 0) return fail(ERI_EINVAL, "output not 8-byte aligned");
  cudaStream_t stream = (cudaStream_t)stream_;
  Library& L = lib();
  const size_t nlaunch = 1 + plan->buckets.size();
  if (plan->timing && plan->events.size() < 2 * nlaunch) {
    for (size_t i = plan->events.size(); i < 2 * nlaunch; ++i) {
      cudaEvent_t e;
      CUDA_OR(cudaEventCreate(&e), "cudaEventCreate");
      plan->events.push_back(e);
    }
  }
  size_t li = 0;
  cudaStream_t cur = stream;  // stream of the current launch
  auto mark = [&](int end) -> cudaError_t {
    return plan->timing ? cudaEventRecord(plan->events[2 * li + end], cur) : cudaSuccess;
  };
  // lanes of the current round that received work, to join back
  std::vector<char> lane_used(plan->nlanes, 0);
  auto join_round = [&]() -> int {
    for (int l = 1; l < plan->nlanes; ++l) {
      if (!lane_used[l]) continue;
      CUDA_OR(cudaEventRecord(plan->join_ev[l - 1], plan->lanes[l - 1]), "cudaEventRecord (join)");
      CUDA_OR(cudaStreamWaitEvent(stream, plan->join_ev[l - 1], 0), "cudaStreamWaitEvent (join)");
      lane_used[l] = 0;
    }
    return ERI_OK;
  };
  int cur_round = -1;
  if (plan->zero_out)
    CUDA_OR(cudaMemsetAsync(out, 0, (size_t)plan->offsets.back() * sizeof(double), stream), "zero output");
  if (fz)
    CUDA_OR(cudaMemsetAsync(plan->done_q.p, 0, plan->done_q.n * sizeof(int32_t), stream), "zero part counters");
  {
    CUDA_OR(mark(0), "cudaEventRecord");
    // molecule plans have their primitive pairs already (npair = 0)
    const int threads = 128;
    const int blocks = (plan->npair + threads - 1) / threads;
    if (blocks > 0) {
      eri_pair_setup_kernel<<<blocks, threads, 0, stream>>>(plan->pin.p, plan->npair, plan->shells.p, plan->exps.p,
                                                            plan->coefs.p, plan->plist.p, plan->pairs.p,
                                                            plan->pprims.p, plan->pprims_f.p);
      CUDA_OR(cudaGetLastError(), "pair set-up launch");
    }
    CUDA_OR(mark(1), "cudaEventRecord");
    ++li;
  }
  for (const Bucket& b : plan->buckets) {
    if (b.round != cur_round) {
      // a round's blocks are complete before the next round adds to them
      if (int rc = join_round()) return rc;
      cur_round = b.round;
      if (plan->nlanes > 1) CUDA_OR(cudaEventRecord(plan->fork_ev, stream), "cudaEventRecord (fork)");
    }
    cur = stream;
    if (b.lane > 0) {
      cur = plan->lanes[b.lane - 1];
      if (!lane_used[b.lane]) {
        CUDA_OR(cudaStreamWaitEvent(cur, plan->fork_ev, 0), "cudaStreamWaitEvent (fork)");
        lane_used[b.lane] = 1;
      }
    }
    CUDA_OR(mark(0), "cudaEventRecord");
    EriLaunchArgs a;
    a.quartets = plan->quartets.p + b.first;
    a.pairs = plan->pairs.p;
    a.pprims = plan->mol ? plan->mol->pprims_d.p : plan->pprims.p;
    a.pprims_f = plan->mol ? plan->mol->pprims_f.p : plan->pprims_f.p;
    a.boys_tab = L.d_boys;
    a.out = out;
    a.scratch = plan->scratch.p;
    a.scratch_stride = plan->scratch_stride;
    a.nq = (int32_t)b.count;
    a.group = b.group;
    if (b.tier == TIER_REG) {
      void* args[] = {&a};
      CUDA_OR(cudaLaunchKernel(b.reg_fn, dim3(b.grid), dim3(b.block), args, 0, cur), "class kernel launch");
    } else if (b.tier == TIER_PERSIST) {
      EriPersistArgs pa;
      pa.items = plan->items.p + b.item0;
      pa.progs = plan->progs.p;
      pa.next = plan->counters.p + b.pgroup;
      pa.nitems = b.nitems;
      pa.pad = 0;
      pa.gH = plan->persist_h.p;
      pa.gh_per_block = plan->persist_h_per_block;
      pa.c2s = L.d_c2s;
      memset(&pa.fuse, 0, sizeof pa.fuse);
      if (fz) {
        pa.fuse.on = 1;
        pa.fuse.jk.quartets = plan->d_uq.p;
        pa.fuse.jk.offsets = plan->d_offsets.p;
        pa.fuse.jk.shell_bf = plan->d_shell_bf.p;
        pa.fuse.jk.blocks = out;
        pa.fuse.jk.D = fz->D;
        pa.fuse.jk.J = fz->J;
        pa.fuse.jk.K = fz->K;
        pa.fuse.jk.nq = plan->nq;
        pa.fuse.jk.nbf = fz->nbf;
        pa.fuse.rec_q = plan->rec_q.p;
        pa.fuse.nparts = plan->nparts_q.p;
        pa.fuse.done = plan->done_q.p;
      }
      a.quartets = plan->quartets.p;  // items index the whole record array
      CUDA_OR(cudaMemsetAsync(pa.next, 0, sizeof(int32_t), cur), "zero item counter");
      CUDA_OR(eri_coop_persist_launch(b.fp32, b.vote, &a, &pa, b.grid, b.smem, cur), "persistent launch");
    } else if (b.tier == TIER_COOP) {
      const CoopProg* cp = b.coop;
      EriCoopArgs p;
      p.ph1 = cp->d_ph1;
      p.steps1 = cp->d_steps1;
      p.ph2 = cp->d_ph2;
      p.steps2 = cp->d_steps2;
      p.c2s = L.d_c2s;
      p.gvals = plan->coop_vals.p;
      p.gH = plan->coop_h.p;
      p.nw1 = cp->nw1;
      p.nw2 = cp->nw2;
      p.nh = cp->nh;
      p.nslot = cp->nslot;
      p.L = cp->L;
      p.smem_slots = b.smem_slots;
      p.h_in_smem = b.h_in_smem;
      p.nteams = b.nteams;
      p.batch = b.batch;
      p.single = b.single;
      CUDA_OR(eri_coop_launch(cp->T, cp->ilp, b.fp32, b.vote, &a, &p, b.grid, b.block, b.smem, cur),
              "cooperative launch");
    } else {
      EriProgArgs p;
      p.ph1 = b.prog->d_ph1;
      p.ph2 = b.prog->d_ph2;
      p.c2s = L.d_c2s;
      p.n1 = b.prog->n1;
      p.n2 = b.prog->n2;
      p.nh = b.prog->nh;
      p.L = b.prog->L;
      CUDA_OR(eri_exec_launch(b.tier == TIER_SHARED, &a, &p, b.grid, b.block, b.smem, cur), "executor launch");
    }
    CUDA_OR(mark(1), "cudaEventRecord");
    ++li;
  }
  return join_round();
}

// The separate digestion kernels over the plan's quartet lists: every quartet
// (rest = false), or the quartets a persistent launch does not digest.
static int digest_lists(eri_plan_t* plan, const double* blocks, const double* density, int32_t nbf, double* J,
                        double* K, void* stream, bool rest) {
  EriDigestArgs g;
  g.quartets = plan->d_uq.p;
  g.offsets = plan->d_offsets.p;
  g.shell_bf = plan->d_shell_bf.p;
  g.blocks = blocks;
  g.D = density;
  g.J = J;
  g.K = K;
  g.nq = plan->nq;
  g.nbf = nbf;
  g.tri = 0;
  // mirrored pairs of J and K entries reduce once into the plan's triangles,
  // which are then added into J and K
  const size_t nn = (size_t)nbf * (size_t)nbf;
  const bool tri = plan->jk_tri.n >= 2 * nn && nn > 0;
  if (tri) {
    CUDA_OR(cudaMemsetAsync(plan->jk_tri.p, 0, 2 * nn * sizeof(double), (cudaStream_t)stream), "zero J/K triangles");
    g.J = J ? plan->jk_tri.p : nullptr;
    g.K = K ? plan->jk_tri.p + nn : nullptr;
    g.tri = 1;
  }
  const DevBuf<int64_t>& sm = rest ? plan->d_rsmall : plan->d_small;
  const DevBuf<int64_t>& lg = rest ? plan->d_rlarge : plan->d_large;
  if (sm.n > 0) {
    g.list = sm.p;
    g.nlist = (int64_t)sm.n;
    CUDA_OR(eri_digest_launch(&g, 1, (cudaStream_t)stream), "digest launch");
  }
  if (lg.n > 0) {
    g.list = lg.p;
    g.nlist = (int64_t)lg.n;
    CUDA_OR(eri_digest_launch(&g, 0, (cudaStream_t)stream), "digest launch");
  }
  if (tri) {
    if (J) CUDA_OR(eri_digest_fold_launch(plan->jk_tri.p, J, nbf, (cudaStream_t)stream), "fold J");
    if (K) CUDA_OR(eri_digest_fold_launch(plan->jk_tri.p + nn, K, nbf, (cudaStream_t)stream), "fold K");
  }
  return ERI_OK;
}

extern "C" int eri_digest_jk(eri_plan_t* plan, const double* blocks, const double* density, int32_t nbf, double* J,
                             double* K, void* stream) {
  if (!plan) return fail(ERI_EINVAL, "NULL plan");
  if (plan->nq == 0) return ERI_OK;
  if (!plan->digest) return fail(ERI_ESTATE, "plan built without opts.digest = 1");
  if (!blocks || !density) return fail(ERI_EINVAL, "NULL blocks or density");
  if (nbf != plan->nbf) return fail(ERI_EINVAL, "nbf does not match the plan's basis functions");
  if (!J && !K) return ERI_OK;
  return digest_lists(plan, blocks, density, nbf, J, K, stream, false);
}

extern "C" int eri_compute_jk(eri_plan_t* plan, const double* density, int32_t nbf, double* J, double* K,
                              void* stream) {
  if (!plan) return fail(ERI_EINVAL, "NULL plan");
  if (plan->nq == 0) return ERI_OK;
  if (!plan->digest) return fail(ERI_ESTATE, "plan built without opts.digest = 1");
  const size_t n = (size_t)plan->offsets.back();
  if (plan->outbuf.n < n) {
    plan->outbuf.reset();
    if (int rc = plan->outbuf.alloc(n, "output buffer")) return rc;
  }
  if (!density) return fail(ERI_EINVAL, "NULL density");
  if (nbf != plan->nbf) return fail(ERI_EINVAL, "nbf does not match the plan's basis functions");
  if (!J && !K) return eri_compute(plan, plan->outbuf.p, stream);
  if (!plan->persistent) {
    // the separate digestion pass after the evaluation.  Digesting each
    // bucket's quartets on its stream right after its launch was measured
    // slower (the 60-atom water cluster: 307.6 ms against 294.4 ms per
    // step): the latency-bound digestion blocks then hold SMs that the
    // concurrent FP64-bound class launches would use.
    if (int rc = eri_compute(plan, plan->outbuf.p, stream)) return rc;
    return digest_lists(plan, plan->outbuf.p, density, nbf, J, K, stream, false);
  }
  // the digestion runs in the evaluation launch itself, then the quartets
  // whose parts all ran on the register tier
  const FuseIn fz = {density, J, K, nbf};
  if (int rc = compute_impl(plan, plan->outbuf.p, stream, &fz)) return rc;
  return digest_lists(plan, plan->outbuf.p, density, nbf, J, K, stream, true);
}

extern "C" int eri_plan_set_timing(eri_plan_t* plan, int enable) {
  if (!plan) return fail(ERI_EINVAL, "NULL plan");
  plan->timing = enable != 0;
  return ERI_OK;
}

extern "C" int eri_plan_launch_count(const eri_plan_t* plan) {
  return plan ? (int)(plan->nq ? 1 + plan->buckets.size() : 0) : 0;
}

extern "C" int eri_plan_launch_info(const eri_plan_t* plan, int i, int32_t* info, double* flops, float* ms) {
  if (!plan || i < 0 || i >= eri_plan_launch_count(plan)) return fail(ERI_EINVAL, "bad launch index");
  int32_t v[8] = {-1, -1, -1, -1, 0, 0, 0, 0};
  double f = 0;
  if (i == 0) {
    v[5] = (plan->npair + 127) / 128;
    v[6] = 128;
    v[7] = plan->npair;
  } else {
    const Bucket& b = plan->buckets[i - 1];
    for (int k = 0; k < 4; ++k) v[k] = b.ls[k];
    v[4] = b.tier;
    v[5] = b.grid;
    v[6] = b.block;
    v[7] = (int32_t)b.count;
    f = b.flops;
  }
  if (info) memcpy(info, v, sizeof v);
  if (flops) *flops = f;
  if (ms) {
    *ms = -1.0f;
    if (plan->timing && plan->events.size() >= (size_t)(2 * i + 2)) {
      cudaError_t e = cudaEventElapsedTime(ms, plan->events[2 * i], plan->events[2 * i + 1]);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ERI_ESTATE, std::string("launch timing not available: ") + cudaGetErrorString(e));
      }
    }
  }
  return ERI_OK;
}

extern "C" int eri_plan_launch_shape(const eri_plan_t* plan, int i, int32_t* info) {
  if (!plan || !info || i < 0 || i >= eri_plan_launch_count(plan)) return fail(ERI_EINVAL, "bad launch index");
  int32_t v[4] = {-1, -1, 0, 0};
  if (i > 0) {
    const Bucket& b = plan->buckets[i - 1];
    if (b.tier == TIER_COOP || (b.tier == TIER_PERSIST && b.coop)) {
      v[0] = b.kind;
      v[1] = b.shape;
      v[2] = b.coop ? b.coop->T : 0;
      v[3] = b.vote ? 2 : 1;
    }
  }
  memcpy(info, v, sizeof v);
  return ERI_OK;
}

extern "C" int eri_compute_host(eri_plan_t* plan, double* host_out, void* stream_) {
  if (!plan) return fail(ERI_EINVAL, "NULL plan");
  if (plan->nq == 0) return ERI_OK;
  if (!host_out) return fail(ERI_EINVAL, "NULL output");
  const size_t n = (size_t)plan->offsets.back();
  if (plan->outbuf.n < n) {
    plan->outbuf.reset();
    int rc = plan->outbuf.alloc(n, "output buffer");
    if (rc) return rc;
  }
  int rc = eri_compute(plan, plan->outbuf.p, stream_);
  if (rc) return rc;
  CUDA_OR(cudaMemcpyAsync(host_out, plan->outbuf.p, n * sizeof(double), cudaMemcpyDeviceToHost,
                          (cudaStream_t)stream_),
          "copy to host");
  return ERI_OK;
}

extern "C" int eri_plan_stats(const eri_plan_t* plan, double* stats, int n) {
  if (!plan || !stats || n < 0) return fail(ERI_EINVAL, "bad argument");
  const double v[8] = {(double)plan->buckets.size(), plan->flops, (double)(plan->scratch.n * sizeof(double)),
                       (double)plan->nq, plan->nprimq, plan->h2d_bytes, plan->flops32, (double)plan->nparts32};
  for (int i = 0; i < n && i < 8; ++i) stats[i] = v[i];
  return ERI_OK;
}

extern "C" int eri_plan_launch_precision(const eri_plan_t* plan, int i) {
  if (!plan || i < 0 || i >= eri_plan_launch_count(plan)) return fail(ERI_EINVAL, "bad launch index");
  return i > 0 && plan->buckets[i - 1].fp32 ? 32 : 64;
}

extern "C" int eri_plan_destroy(eri_plan_t* plan) {
  if (!plan) return ERI_OK;
  // a stream-ordered plan frees its memory on its stream, after the work
  // already queued there; any other plan waits for the device first
  if (!plan->stream_ordered) cudaDeviceSynchronize();
  delete plan;
  return ERI_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free evaluation (eri_compute_fixed_scratch)
//
// Some callers must not allocate device memory when they evaluate: code whose
// device memory is budgeted and owned by another framework (an application
// that hands out all of the device memory up front), or a latency-critical
// loop that must not enter the allocator (cudaMalloc and cudaFree can
// synchronise the device).  For them the global-scratch program tier can take its
// per-thread value slots from this fixed array instead of the plan's
// scratch.  The array is a file-scope device variable: every GPU that loads
// the library holds its 64 MiB until the process exits.
// ---------------------------------------------------------------------------
#define ERI_FIXED_SCRATCH_DOUBLES (8u * 1024u * 1024u)  // 64 MiB
static __device__ __align__(256) double eri_fixed_scratch[ERI_FIXED_SCRATCH_DOUBLES];

namespace {
// Device address of eri_fixed_scratch, looked up once per device with that
// device current (host code may not use the symbol's name as an address).
int fixed_scratch_ptr(double** out) {
  static std::mutex mu;
  static std::map<int, double*> ptrs;
  int dev = 0;
  CUDA_OR(cudaGetDevice(&dev), "cudaGetDevice");
  std::lock_guard<std::mutex> g(mu);
  auto it = ptrs.find(dev);
  if (it == ptrs.end()) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, eri_fixed_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(ERI_ECUDA, std::string("cudaGetSymbolAddress(eri_fixed_scratch): ") + cudaGetErrorString(e));
    it = ptrs.emplace(dev, (double*)p).first;
  }
  *out = it->second;
  return ERI_OK;
}
}  // namespace

extern "C" int eri_compute_fixed_scratch(eri_plan_t* plan, double* out, void* stream_) {
  if (!plan) return fail(ERI_EINVAL, "NULL plan");
  if (plan->nq == 0) return ERI_OK;
  if (!out) return fail(ERI_EINVAL, "NULL output");
  if (((uintptr_t)out & 7) != 0) return fail(ERI_EINVAL, "output not 8-byte aligned");
  for (const Bucket& b : plan->buckets) {
    if (b.tier != TIER_GLOBAL)
      return fail(ERI_EUNSUPPORTED, "eri_compute_fixed_scratch needs a plan built with tier = 3 (global scratch)");
    // one block of 128 threads must fit: nslot * 128 doubles
    if ((size_t)b.prog->nslot * 128 > ERI_FIXED_SCRATCH_DOUBLES)
      return fail(ERI_EINVAL, "class (" + std::to_string(b.ls[0]) + std::to_string(b.ls[1]) + "|" +
                                  std::to_string(b.ls[2]) + std::to_string(b.ls[3]) + ") needs " +
                                  std::to_string((size_t)b.prog->nslot * 128 * 8) +
                                  " bytes of scratch per 128-thread block; the fixed scratch holds " +
                                  std::to_string((size_t)ERI_FIXED_SCRATCH_DOUBLES * 8));
  }
  double* scratch = nullptr;
  int rc = fixed_scratch_ptr(&scratch);
  if (rc) return rc;
  cudaStream_t stream = (cudaStream_t)stream_;
  Library& L = lib();
  // parts that add into their block need it zeroed first (a memset
  // allocates nothing)
  if (plan->zero_out)
    CUDA_OR(cudaMemsetAsync(out, 0, (size_t)plan->offsets.back() * sizeof(double), stream), "zero output");
  {
    // molecule plans have their primitive pairs already (npair = 0)
    const int threads = 128;
    const int blocks = (plan->npair + threads - 1) / threads;
    if (blocks > 0) {
      eri_pair_setup_kernel<<<blocks, threads, 0, stream>>>(plan->pin.p, plan->npair, plan->shells.p, plan->exps.p,
                                                            plan->coefs.p, plan->plist.p, plan->pairs.p,
                                                            plan->pprims.p, plan->pprims_f.p);
      CUDA_OR(cudaGetLastError(), "pair set-up launch");
    }
  }
  for (const Bucket& b : plan->buckets) {
    // as many 128-thread blocks as the fixed array holds, at most the plan's
    // grid; the executor strides over the remaining quartets
    const int fit = (int)(ERI_FIXED_SCRATCH_DOUBLES / ((size_t)b.prog->nslot * 128));
    const int grid = std::max(1, std::min(b.grid, fit));
    EriLaunchArgs a;
    a.quartets = plan->quartets.p + b.first;
    a.pairs = plan->pairs.p;
    a.pprims = plan->mol ? plan->mol->pprims_d.p : plan->pprims.p;
    a.pprims_f = plan->mol ? plan->mol->pprims_f.p : plan->pprims_f.p;
    a.boys_tab = L.d_boys;
    a.out = out;
    a.scratch = scratch;
    a.scratch_stride = (int64_t)grid * 128;
    a.nq = (int32_t)b.count;
    a.group = b.group;
    EriProgArgs p;
    p.ph1 = b.prog->d_ph1;
    p.ph2 = b.prog->d_ph2;
    p.c2s = L.d_c2s;
    p.n1 = b.prog->n1;
    p.n2 = b.prog->n2;
    p.nh = b.prog->nh;
    p.L = b.prog->L;
    CUDA_OR(eri_exec_launch(0, &a, &p, grid, 128, 0, stream), "executor launch (fixed scratch)");
  }
  return ERI_OK;
}

// ---------------------------------------------------------------------------
// Diagnostic: the device Boys function on its own
// ---------------------------------------------------------------------------
// The compiled register-tier kernels inline eri_boys<L> with a compile-time
// order; one instantiation per order.
template <int L>
__global__ void eri_boys_reg_kernel(const double* __restrict__ T, int64_t n, const double* __restrict__ tab,
                                    double* __restrict__ F) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double f[L + 1];
  eri_boys<L>(T[i], f, tab);
#pragma unroll
  for (int m = 0; m <= L; ++m) F[i * (L + 1) + m] = f[m];
}

template <int L>
static cudaError_t boys_reg_launch(const double* T, int64_t n, int l, const double* tab, double* F, cudaStream_t st) {
  if (l != L) return boys_reg_launch<(L < ERI_BOYS_LMAX ? L + 1 : L)>(T, n, l, tab, F, st);
  eri_boys_reg_kernel<L><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(T, n, tab, F);
  return cudaGetLastError();
}

extern "C" int eri_boys_eval(const double* T, int64_t n, int32_t L, int32_t form, double* F, void* stream_) {
  if (n < 0 || L < 0 || L > ERI_BOYS_LMAX || form < 0 || form > 2) return fail(ERI_EINVAL, "bad n, L or form");
  if (n == 0) return ERI_OK;
  if (!T || !F) return fail(ERI_EINVAL, "NULL argument");
  int rc = ensure_library();
  if (rc) return rc;
  const double* tab = lib().d_boys;
  cudaStream_t st = (cudaStream_t)stream_;
  cudaError_t e = form == 0   ? boys_reg_launch<0>(T, n, L, tab, F, st)
                  : form == 1 ? eri_coop_boys_launch(T, n, L, tab, F, st)
                              : eri_exec_boys_launch(T, n, L, tab, F, st);
  CUDA_OR(e, "Boys launch");
  return ERI_OK;
}

// ---------------------------------------------------------------------------
// Schwarz bounds, tier table, CUDA-graph replay
// ---------------------------------------------------------------------------
// Q_q = sqrt(max_i |block_q[i, i]|) over the (ab|ab)-shaped block of quartet
// q (the diagonal of the n_ab x n_ab matrix): the Schwarz factor of pair ab,
// |(ab|cd)| <= Q_ab Q_cd.
__global__ void eri_schwarz_kernel(const double* __restrict__ blocks, const int64_t* __restrict__ off,
                                   const int32_t* __restrict__ nab, int64_t nq, double* __restrict__ q) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  const double* b = blocks + off[i];
  const int n = nab[i];
  double m = 0.0;
  for (int k = 0; k < n; ++k) m = fmax(m, fabs(b[(int64_t)k * n + k]));
  q[i] = sqrt(m);
}

extern "C" int eri_schwarz(const eri_plan_t* plan, const double* blocks, double* bounds, void* stream_) {
  if (!plan || !blocks || !bounds) return fail(ERI_EINVAL, "NULL argument");
  const int64_t nq = plan->nq;
  if (nq == 0) return ERI_OK;
  if (plan->nab.empty()) return fail(ERI_EINVAL, "plan is not made of (ab|ab) quartets");
  cudaStream_t stream = (cudaStream_t)stream_;
  const int threads = 256;
  eri_schwarz_kernel<<<(unsigned)((nq + threads - 1) / threads), threads, 0, stream>>>(
      blocks, plan->d_offsets.p, plan->d_nab.p, nq, bounds);
  CUDA_OR(cudaGetLastError(), "schwarz launch");
  return ERI_OK;
}

extern "C" cudaError_t eri_screen_count_launch(const double* Q, int64_t npair, double t, int64_t* cnt, int64_t* off,
                                               cudaStream_t stream);
extern "C" cudaError_t eri_screen_write_launch(const double* Q, const int32_t* pairs, int64_t npair, double t,
                                               const int64_t* off, int32_t* out, cudaStream_t stream);

extern "C" int eri_screen_quartets(const double* Q, const int32_t* pairs, int64_t npair, double threshold,
                                   int32_t* out, int64_t max_out, int64_t* count, void* stream_) {
  if (!count || npair < 0 || (npair > 0 && (!Q || !pairs)) || std::isnan(threshold))
    return fail(ERI_EINVAL, "bad argument");
  *count = 0;
  if (npair == 0) return ERI_OK;
  if (((uintptr_t)Q & 7) || ((uintptr_t)pairs & 7) || (out && ((uintptr_t)out & 15)))
    return fail(ERI_EINVAL, "Q and pairs must be 8-byte aligned, out 16-byte aligned");
  cudaStream_t stream = (cudaStream_t)stream_;
  int64_t* tmp = nullptr;  // counts [npair], offsets [npair + 1]
  CUDA_OR(cudaMallocAsync((void**)&tmp, (size_t)(2 * npair + 1) * sizeof(int64_t), stream), "screening scratch");
  int64_t total = 0;
  cudaError_t e = eri_screen_count_launch(Q, npair, threshold, tmp, tmp + npair, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&total, tmp + 2 * npair, sizeof(int64_t), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  int rc = ERI_OK;
  if (e != cudaSuccess) {
    rc = fail(ERI_ECUDA, std::string("screening: ") + cudaGetErrorString(e));
  } else {
    *count = total;
    if (out) {
      if (total > max_out) {
        rc = fail(ERI_EINVAL, "out holds " + std::to_string(max_out) + " quartets, " + std::to_string(total) +
                                  " survive");
      } else {
        e = eri_screen_write_launch(Q, pairs, npair, threshold, tmp + npair, out, stream);
        if (e != cudaSuccess) rc = fail(ERI_ECUDA, std::string("screening write: ") + cudaGetErrorString(e));
      }
    }
  }
  cudaFreeAsync(tmp, stream);
  return rc;
}

namespace {
std::mutex g_tier_mu;
std::map<std::vector<int>, int> g_tier_table;  // class -> preferred tier (autotuner)
}  // namespace

extern "C" int eri_set_class_tier(int la, int lb, int lc, int ld, int tier) {
  if (la < 0 || lb < 0 || lc < 0 || ld < 0 || la > ERI_MAX_L || lb > ERI_MAX_L || lc > ERI_MAX_L ||
      ld > ERI_MAX_L || tier < 0 || tier > 4)
    return fail(ERI_EINVAL, "bad class or tier");
  std::lock_guard<std::mutex> g(g_tier_mu);
  if (tier == 0)
    g_tier_table.erase({la, lb, lc, ld});
  else
    g_tier_table[{la, lb, lc, ld}] = tier;
  return ERI_OK;
}

int preferred_tier(const int ls[4]) {
  std::lock_guard<std::mutex> g(g_tier_mu);
  auto it = g_tier_table.find({ls[0], ls[1], ls[2], ls[3]});
  return it == g_tier_table.end() ? 0 : it->second;
}

namespace {
std::map<std::vector<int>, int> g_vote_table;  // class -> preferred vote form (autotuner)
}  // namespace

extern "C" int eri_set_class_votes(int la, int lb, int lc, int ld, int votes) {
  if (la < 0 || lb < 0 || lc < 0 || ld < 0 || la > ERI_MAX_L || lb > ERI_MAX_L || lc > ERI_MAX_L ||
      ld > ERI_MAX_L || votes < 0 || votes > 2)
    return fail(ERI_EINVAL, "bad class or vote form");
  std::lock_guard<std::mutex> g(g_tier_mu);
  if (votes == 0)
    g_vote_table.erase({la, lb, lc, ld});
  else
    g_vote_table[{la, lb, lc, ld}] = votes;
  return ERI_OK;
}

int preferred_votes(const int ls[4]) {
  std::lock_guard<std::mutex> g(g_tier_mu);
  auto it = g_vote_table.find({ls[0], ls[1], ls[2], ls[3]});
  return it == g_vote_table.end() ? 0 : it->second;
}

namespace {
// (class, kind) -> (shape index, vote form) (autotuner)
std::map<std::vector<int>, std::pair<int, int>> g_shape_table;
}  // namespace

extern "C" int eri_set_class_shape(int la, int lb, int lc, int ld, int kind, int shape, int votes) {
  if (la < 0 || lb < 0 || lc < 0 || ld < 0 || la > ERI_MAX_L || lb > ERI_MAX_L || lc > ERI_MAX_L ||
      ld > ERI_MAX_L || kind < 0 || kind > 2 || shape < -1 || votes < 0 || votes > 2)
    return fail(ERI_EINVAL, "bad class, kind, shape or vote form");
  std::lock_guard<std::mutex> g(g_tier_mu);
  if (shape < 0)
    g_shape_table.erase({la, lb, lc, ld, kind});
  else
    g_shape_table[{la, lb, lc, ld, kind}] = {shape, votes};
  return ERI_OK;
}

bool preferred_shape(const int ls[4], int kind, int* shape, int* votes) {
  std::lock_guard<std::mutex> g(g_tier_mu);
  auto it = g_shape_table.find({ls[0], ls[1], ls[2], ls[3], kind});
  if (it == g_shape_table.end()) return false;
  *shape = it->second.first;
  *votes = it->second.second;
  return true;
}

extern "C" int eri_class_shapes(int la, int lb, int lc, int ld, int32_t* info, int max) {
  if (la < 0 || lb < 0 || lc < 0 || ld < 0 || la > ERI_MAX_L || lb > ERI_MAX_L || lc > ERI_MAX_L ||
      ld > ERI_MAX_L || max < 0 || (max > 0 && !info))
    return fail(ERI_EINVAL, "bad class or output");
  int rc = ensure_library();
  if (rc) return rc;
  Library& L = lib();
  const std::vector<CoopProg*> v = class_shapes(L, {la, lb, lc, ld, 0, 0, 0});
  for (int i = 0; i < (int)v.size() && i < max; ++i) {
    const CoopProg* p = v[i];
    const int32_t e[5] = {p->T, p->ilp, p->k1, p->k2, p->nslot};
    memcpy(info + 5 * i, e, sizeof e);
  }
  return (int)v.size();
}

// Capture run(stream) -- eri_compute or eri_compute_jk of the plan -- into
// the plan's graph.
template <typename Run>
static int graph_capture(eri_plan_t* plan, void* stream_, Run run) {
  if (!plan) return fail(ERI_EINVAL, "NULL plan");
  cudaStream_t stream = (cudaStream_t)stream_;
  if (stream == nullptr) return fail(ERI_EINVAL, "capture needs a non-default stream");
  if (plan->graph_exec) {
    cudaGraphExecDestroy(plan->graph_exec);
    plan->graph_exec = nullptr;
  }
  const bool timing = plan->timing;
  plan->timing = false;
  CUDA_OR(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  const int rc = run(stream_);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(stream, &graph);
  plan->timing = timing;
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return fail(ERI_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&plan->graph_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(ERI_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  return ERI_OK;
}

extern "C" int eri_plan_graph_capture(eri_plan_t* plan, double* out, void* stream) {
  return graph_capture(plan, stream, [&](void* st) { return eri_compute(plan, out, st); });
}

extern "C" int eri_plan_graph_capture_jk(eri_plan_t* plan, const double* density, int32_t nbf, double* J, double* K,
                                         void* stream) {
  if (plan && plan->nq > 0 && plan->digest && (size_t)plan->offsets.back() > plan->outbuf.n) {
    // the plan's block buffer is allocated before the capture, not inside it
    plan->outbuf.reset();
    if (int rc = plan->outbuf.alloc((size_t)plan->offsets.back(), "output buffer")) return rc;
  }
  return graph_capture(plan, stream, [&](void* st) { return eri_compute_jk(plan, density, nbf, J, K, st); });
}

extern "C" int eri_plan_graph_launch(eri_plan_t* plan, void* stream_) {
  if (!plan || !plan->graph_exec) return fail(ERI_ESTATE, "no captured graph (call eri_plan_graph_capture)");
  CUDA_OR(cudaGraphLaunch(plan->graph_exec, (cudaStream_t)stream_), "cudaGraphLaunch");
  return ERI_OK;
}
