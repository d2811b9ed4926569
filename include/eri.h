/*
 * eri.h -- C ABI of the GB300 contracted-ERI engine.
 *
 * The library evaluates contracted Gaussian electron repulsion integrals
 * (ab|cd) (FusionRCG paper, Sec. II-A, Eq. 1) by the Head-Gordon-Pople
 * scheme: Boys function and Obara-Saika vertical recurrence per primitive
 * quartet (Eq. 2), contraction, horizontal recurrence (Eq. 3) with the
 * Cartesian-to-spherical transform fused stepwise (Eqs. 8, 16).  The
 * arithmetic is FP64 (eri_plan_mixed: FP32 recurrences for quartets whose
 * bound is below a threshold) and runs in CUDA kernels for sm_103a.
 *
 * Conventions (bohr, Hartree atomic units):
 *  - a primitive x^i y^j z^k exp(-a r^2) of shell angular momentum l carries
 *    N(a, l) = (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2l-1)!!); contraction
 *    coefficients are used as given (no renormalisation);
 *  - Cartesian components in x-descending, then y-descending order
 *    (xx, xy, xz, yy, yz, zz);
 *  - spherical components: real solid harmonics, Racah normalised, no
 *    Condon-Shortley phase, m = -l..l (so p is ordered y, z, x);
 *  - the block of quartet (s0 s1 | s2 s3) is row-major over the components
 *    of s0, s1, s2, s3 in that order; blocks follow the quartet list.
 *
 * Errors: every call returns ERI_OK (0) or a negative ERI_E* code;
 * eri_last_error() gives a message for the calling thread's last failure.
 * Plans are not thread-safe: one thread at a time may use a plan, and one
 * eri_compute per plan may be in flight (the plan's device buffers are
 * reused by the next call).
 */
#ifndef ERI_H
#define ERI_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ERI_OK = 0,
  ERI_EINVAL = -1,        /* bad argument: l, K, index, non-positive or non-finite exponent */
  ERI_EUNSUPPORTED = -2,  /* l > 4, or a tier/option combination that is not built */
  ERI_ENOMEM = -3,        /* device or host allocation failed */
  ERI_ECUDA = -4,         /* a CUDA call failed (message in eri_last_error) */
  ERI_EBUSY = -5,         /* reserved: plan in use */
  ERI_ETIMEOUT = -6,      /* a bounded wait expired (serving waits) */
  ERI_ESTATE = -7         /* library files missing or inconsistent */
};

/* One contracted shell: angular momentum l (0..4), contraction depth nprim
 * (1..ERI_MAX_NPRIM), index of its centre, offset of its first primitive in
 * the exponent/coefficient arrays. */
typedef struct {
  int32_t l;
  int32_t nprim;
  int32_t center;
  int32_t prim_offset;
} eri_shell;

#define ERI_MAX_L 4
#define ERI_MAX_NPRIM 32

/* Basis data, host memory, read during eri_plan only (copied). */
typedef struct {
  const double* centers;    /* [ncenter][3], bohr */
  int32_t ncenter;
  const double* exponents;  /* [nprim_total], > 0 */
  const double* coefs;      /* [nprim_total], raw contraction coefficients */
  int32_t nprim_total;
} eri_basis;

/* Plan options; pass NULL for the defaults (all zero). */
typedef struct {
  int32_t axis_rule;    /* 0 consumer-first z->y->x (Sec. III-A), 1 Algorithm 1 as printed, 2 bra-first x->y->z */
  int32_t schedule;     /* 0 DSA (Eq. 7), 1 level order (no DSA) */
  int32_t sph_mode;     /* 0 stepwise fusion (Eq. 16), 1 materialize-then-transform (Eq. 17), 2 Cartesian output */
  int32_t tier;         /* 0 auto, 1 register (compiled), 2 shared-memory program, 3 global-scratch program,
                           4 team-cooperative program (values shared by a team of lanes) */
  int32_t orientation;  /* 0 per primitive pair: each recurs on its tighter primitive's centre (a pair may split
                           into two oriented parts whose blocks are summed), 1 whole pair on the higher l,
                           2 whole pair on the shell holding the largest exponent */
  int32_t streams;      /* launches of one part round that may run concurrently, on up to this many streams
                           (the caller's plus streams the plan owns, joined back before eri_compute returns):
                           0 auto (4 for plans holding several classes, else 1), 1 serial, at most 8 */
  int32_t digest;       /* 1: also keep on the device what eri_digest_jk / eri_compute_jk need (the quartet list,
                           16 B per quartet, digestion lists, and the J/K triangles, 2 nbf^2 doubles when at
                           most 1 GiB); 0: no */
  int32_t votes;        /* team-cooperative tier: 0 auto (the class table of eri_set_class_votes, else on for
                           teams of 128 lanes or more), 1 each lane predicates its optional FP64 terms, 2 each
                           optional term sits behind a warp vote */
  int32_t persistent;   /* 1: every class without a compiled register-tier kernel (with tier 4: every class) in
                           one persistent launch per precision and vote form over a device work list (one
                           512-thread block per SM takes items -- runs of one class's quartets -- from a
                           counter); the parts of a quartet reduce into its zeroed block in any order; tier
                           must be 0 or 4.  0: one launch per class bucket */
  int32_t ordered;      /* a quartet evaluated in several parts (the two orientations of a split shell pair,
                           chunks of a deep contraction): 0: every part runs in the same launch round and
                           reduces into the quartet's zeroed block with FP64 atomic additions, so the last bits
                           of such blocks depend on the order of the additions; 1: part k runs in launch round
                           k and adds into the block in that order (bitwise reproducible for quartets whose
                           parts are not chunked; more launches, each round joined before the next).  Chunks
                           of one part reduce atomically either way.  A persistent plan takes 0 */
} eri_opts;

typedef struct eri_plan_s eri_plan_t;
typedef struct eri_mol_s eri_mol_t;

/* Build a plan for nq shell quartets (quartets = [nq][4] shell indices, any
 * order, host memory).  What the plan evaluates is the contracted integral
 * (ab|cd) of Sec. II-A, Eq. 1, by the steps of Algorithm 2: per primitive
 * pair the Gaussian-product data (zeta, P, K_AB), per primitive quartet the
 * Boys function and the vertical recurrence of Eq. 2 (and its ket mirror) in
 * the axis order of Algorithm 1 and the DSA order of Eq. 7, contraction into
 * the accumulator bank, then per shell quartet the horizontal recurrence of
 * Eq. 3 with the spherical transform fused stepwise (Sec. III-B, Eq. 16).
 * Validates every input, canonicalises each quartet to
 * its class and orientation, uploads basis, pair list and quartet records to
 * the current CUDA device and sizes the scratch.  Host inputs are copied;
 * the plan owns its device memory.  nq may be 0, and is at most 2^31 - 1
 * (ERI_EINVAL above).  Synchronous. */
int eri_plan(const eri_shell* shells, int32_t nshell, const eri_basis* basis, const int32_t* quartets,
             int64_t nq, const eri_opts* opts, eri_plan_t** plan_out);

/* Mixed-precision plan (the precision axis of the method's extensions; the
 * paper evaluates everything in FP64 and has no counterpart).  Like eri_plan,
 * plus qbound (host, nq doubles >= 0): an upper bound on |(ab|cd)| for each
 * quartet, normally the Schwarz product Q_ab Q_cd.  Quartets with
 * qbound[q] < fp32_below run the primitive-quartet set-up (W - P, W - Q, T,
 * the prefactor and the recurrence coefficients, from an FP32 copy of the
 * primitive-pair data) and the recurrences (VRR, contraction sums, HRR and
 * the spherical transform) in FP32; the Boys function, every other quartet
 * and the output (stores and the accumulation of split parts) stay FP64.  The absolute error of an FP32
 * quartet is then about qbound[q] times a small multiple of 2^-24 per
 * recurrence level.  FP32 is used only with the default generator options
 * and tier 0, 1 or 4; otherwise the plan is all FP64.  Errors: ERI_EINVAL
 * for a NULL bound array (nq > 0), a negative or NaN bound, or a negative or
 * non-finite threshold; otherwise as eri_plan. */
int eri_plan_mixed(const eri_shell* shells, int32_t nshell, const eri_basis* basis, const int32_t* quartets,
                   int64_t nq, const double* qbound, double fp32_below, const eri_opts* opts,
                   eri_plan_t** plan_out);

/* Stream-ordered plan, for serving loops whose requests overlap on the
 * device: like eri_plan_mixed (qbound may be NULL: all FP64), but every
 * device buffer of the plan is allocated with cudaMallocAsync and filled
 * with cudaMemcpyAsync on stream (a non-default cudaStream_t), and
 * eri_plan_destroy frees them with cudaFreeAsync on the same stream instead
 * of synchronising the device.  Run eri_compute for this plan on the same
 * stream (or on one ordered after it) and destroy the plan only after the
 * last eri_compute was enqueued.  Host inputs are copied before the call
 * returns.  Errors: ERI_EINVAL for a NULL stream or bad bounds; otherwise as
 * eri_plan. */
int eri_plan_on_stream(const eri_shell* shells, int32_t nshell, const eri_basis* basis, const int32_t* quartets,
                       int64_t nq, const double* qbound, double fp32_below, const eri_opts* opts, void* stream,
                       eri_plan_t** plan_out);

/* A molecule kept on the device, for many plans over the same basis (a
 * serving loop's registered molecules): validates and copies the shells and
 * basis, orients every shell pair a >= b (opts->orientation; the other
 * options are ignored) and computes all of their primitive-pair records
 * once on the device.  Synchronous; the handle owns its device memory
 * (about 72 B per primitive pair of the basis).  Errors as eri_plan. */
int eri_mol_create(const eri_shell* shells, int32_t nshell, const eri_basis* basis, const eri_opts* opts,
                   eri_mol_t** mol_out);

/* Release a molecule (synchronises the device first).  Plans built on it
 * must have been destroyed before. */
int eri_mol_destroy(eri_mol_t* mol);

/* A plan over a molecule's shells (quartets index its shells): like
 * eri_plan_mixed (qbound may be NULL: all FP64), but the plan uses the
 * molecule's primitive-pair records instead of building its own, so its
 * construction touches only its quartets and eri_compute launches no pair
 * set-up.  stream: NULL for ordinary allocation, else stream-ordered as in
 * eri_plan_on_stream.  opts->orientation must equal the molecule's.  The
 * plan must not outlive the molecule.  Errors as eri_plan_mixed. */
int eri_plan_on_mol(const eri_mol_t* mol, const int32_t* quartets, int64_t nq, const double* qbound,
                    double fp32_below, const eri_opts* opts, void* stream, eri_plan_t** plan_out);

/* Total number of doubles eri_compute writes (sum of block sizes). */
int64_t eri_output_count(const eri_plan_t* plan);

/* offsets[q] = first element of quartet q's block, offsets[nq] = total;
 * offsets is a host array of nq + 1 int64. */
int eri_output_offsets(const eri_plan_t* plan, int64_t* offsets);

/* Evaluate every quartet of the plan into out (device memory, at least
 * eri_output_count doubles, 8-byte aligned): the blocks (ab|cd) of Eq. 1 as
 * Algorithm 2 computes them, minus its J/K scatter (see eri_digest_jk), with
 * the final transform of Eq. 16 (or Eq. 17 / Cartesian per opts.sph_mode).
 * Asynchronous on stream
 * (a cudaStream_t; NULL = the legacy default stream).  Kernel launch errors
 * are returned; the caller synchronises the stream to observe completion. */
int eri_compute(eri_plan_t* plan, double* out, void* stream);

/* eri_compute into a plan-owned device buffer followed by an asynchronous
 * copy to host_out (host memory, pinned for a truly asynchronous copy, at
 * least eri_output_count doubles) on the same stream. */
int eri_compute_host(eri_plan_t* plan, double* host_out, void* stream);

/* Per-plan statistics, host memory: stats[0] = number of class launches,
 * stats[1] = algorithmic FP64 flops of one eri_compute (FMA = 2),
 * stats[2] = scratch bytes, stats[3] = quartets, stats[4] = primitive
 * quartets, stats[5] = bytes eri_plan copied host-to-device, stats[6] =
 * algorithmic FP32 flops (eri_plan_mixed), stats[7] = quartet parts with
 * FP32 recurrences.  n = entries wanted (<= 8). */
int eri_plan_stats(const eri_plan_t* plan, double* stats, int n);

/* Launch timing: when enabled, eri_compute records a CUDA event pair on its
 * stream around each of its launches (launch 0 = pair set-up, then one per
 * class bucket). */
int eri_plan_set_timing(eri_plan_t* plan, int enable);

/* Number of kernel launches one eri_compute makes (0 for an empty plan). */
int eri_plan_launch_count(const eri_plan_t* plan);

/* Launch i of the last eri_compute: info[8] = {la, lb, lc, ld, tier, grid,
 * block, quartets} (-1 for the pair set-up), *flops = its algorithmic FP64
 * flops, *ms = its duration from the event pair (-1 when timing is off);
 * the stream must have completed.  Any output pointer may be NULL. */
int eri_plan_launch_info(const eri_plan_t* plan, int i, int32_t* info, double* flops, float* ms);

/* Precision of launch i's recurrences: 64, or 32 for an FP32 bucket of an
 * eri_plan_mixed plan (its flops from eri_plan_launch_info are FP32 flops);
 * ERI_EINVAL for a bad index. */
int eri_plan_launch_precision(const eri_plan_t* plan, int i);

/* Coulomb and exchange digestion (FusionRCG Alg. 2, the scatter of each
 * quartet's integrals into the Fock build):
 *     J_ij += sum_kl (ij|kl) D_kl,     K_ij += sum_kl (ik|jl) D_kl
 * from the blocks eri_compute wrote for this plan (device memory, the plan's
 * layout), for a symmetric density D (device, [nbf][nbf] row-major FP64).
 * Each quartet of the plan stands for its orbit under the 8 index
 * permutations: pass every such orbit once (e.g. a >= b, c >= d, pair (ab) >=
 * pair (cd)); quartets that map onto themselves under some permutations are
 * weighted accordingly.  J and K (device, [nbf][nbf], either may be NULL) are
 * accumulated into, not overwritten, with FP64 atomic additions (so the last
 * bits depend on the order of the additions).  nbf must equal the number of
 * basis functions of the plan's shells (spherical, or Cartesian with
 * sph_mode 2), shells numbered consecutively.  The plan must have been built
 * with opts.digest = 1.  Asynchronous on stream.  Each mirrored pair of J (or
 * K) entries receives one reduction, into a plan-owned triangle (2 nbf^2
 * doubles, allocated with the plan when at most 1 GiB) that is then added
 * into J and K on the same stream; digestions of one plan must therefore not
 * overlap on different streams.  Errors: ERI_EINVAL (NULL blocks or density,
 * wrong nbf), ERI_ESTATE (plan without digest data). */
int eri_digest_jk(eri_plan_t* plan, const double* blocks, const double* density, int32_t nbf, double* J,
                  double* K, void* stream);

/* eri_compute into a plan-owned device buffer followed by eri_digest_jk on
 * the same stream: J and K of a density without handing the blocks out.  For
 * a persistent plan (opts.persistent = 1 and opts.digest = 1) the digestion
 * is fused into the evaluation launch: the team that completes a quartet's
 * last part digests its block while it is in L2 (the block is still written
 * to the plan's buffer). */
int eri_compute_jk(eri_plan_t* plan, const double* density, int32_t nbf, double* J, double* K, void* stream);

/* Evaluate like eri_compute without allocating: for callers that may not
 * allocate device memory while they evaluate (a device-memory budget owned
 * by another framework, or a latency-critical loop that must not enter the
 * allocator, which can synchronise the device).  The paper has no
 * counterpart; this is a deployment entry point.  The plan must have been
 * built with opts.tier = 3 (global-scratch program tier); its kernels then
 * take their per-thread value slots from a
 * fixed 64 MiB device array that the library holds on every GPU that loads it
 * until the process exits, so the call itself performs no cudaMalloc,
 * cudaFree or other allocation.  Inputs are the plan's device data, out is
 * the caller's device buffer as for eri_compute.
 *  - Sizes: a class needing more than 64 MiB for one 128-thread block
 *    (nslot x 128 x 8 bytes) is rejected with ERI_EINVAL; otherwise the grid
 *    is reduced to what the array holds, and the kernels stride over the
 *    remaining quartets (slower, same results).
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - Every call shares the one array and the kernels reinitialise what they
 *    read (accumulators are zeroed per quartet; a plan whose parts add into
 *    their blocks has out zeroed first, by a memset), so nothing is carried
 *    between calls; calls that overlap on the GPU (other streams, other
 *    host threads) race on the array and must be serialised by the caller.
 * Returns ERI_EUNSUPPORTED for a plan with non-global tiers. */
int eri_compute_fixed_scratch(eri_plan_t* plan, double* out, void* stream);

/* Schwarz factors.  For a plan whose every quartet is of the form (ab|ab),
 * after eri_compute wrote its blocks to `blocks` (device): bounds[q] =
 * sqrt(max_i |(ab|ab)_ii|) (device, nq doubles), the factor Q_ab of the
 * Cauchy-Schwarz bound |(ab|cd)| <= Q_ab Q_cd used to screen quartet lists.
 * Asynchronous on stream.  ERI_EINVAL for other plans. */
int eri_schwarz(const eri_plan_t* plan, const double* blocks, double* bounds, void* stream);

/* Schwarz screening of the unique quartet list on the device (the batched
 * workload's survivor list).  |(ab|cd)| <= Q_ab Q_cd (Cauchy-Schwarz for the
 * ERI inner product of Eq. 1) with the pair factors Q_ab = sqrt(max|(ab|ab)|)
 * of eri_schwarz.  Q: device [npair] factors; pairs: device [npair][2] shell
 * indices of each pair (8-byte aligned).  The unique quartets are the
 * unordered pairs {P, R} of pairs, P = R included; with lo the pair of the
 * smaller factor (the larger index among equal factors) and hi the other,
 * a quartet survives iff Q_hi >= threshold / Q_lo (Q_lo = 0: iff
 * threshold <= 0).  out: device [max_out][4] int32, 16-byte aligned, or
 * NULL to count only; survivors are written as (P.a, P.b, R.a, R.b), P the
 * larger pair index, ordered by P then R (pairs given in order of falling
 * factor give the sorted-prefix enumeration's list).  *count (host) receives the
 * number of survivors.  Counts on the device (a prefix sum), reads the total
 * back (the stream is synchronised), then writes; temporary device memory
 * is taken stream-ordered and released.  ERI_EINVAL if out is not NULL and
 * max_out < *count (nothing is written). */
int eri_screen_quartets(const double* Q, const int32_t* pairs, int64_t npair, double threshold, int32_t* out,
                        int64_t max_out, int64_t* count, void* stream);

/* Preferred tier for a class (la lb | lc ld) when a plan asks for tier 0:
 * written by the autotuner (paper_2605_10312_gb300.tune); 0 clears the
 * entry.  A preference a class cannot honour falls back to the static rule.
 * Applies to plans built afterwards, process-wide. */
int eri_set_class_tier(int la, int lb, int lc, int ld, int tier);

/* Preferred form of the team-cooperative program for a class (la lb | lc ld)
 * where a plan leaves eri_opts.votes at 0 (auto): 1 optional FP64 terms
 * predicated per lane, 2 skipped by warp vote; 0 clears the entry (written by
 * the autotuner).  Applies to plans built afterwards, process-wide. */
int eri_set_class_votes(int la, int lb, int lc, int ld, int votes);

/* The team-cooperative shapes the build ships for a class (la lb | lc ld)
 * under the default options: entry 0 is the shape taken for deep
 * contractions, then the shape for shallow ones when it differs, then the
 * alternatives an autotuner may time against them.  Each entry is five
 * int32: team lanes T, nodes per lane per step, steps per Phase-1 wave,
 * steps per Phase-2 wave, value slots.  Writes min(count, max) entries to
 * info (host memory, 5 * max int32) and returns the count (0: the class has
 * no cooperative program), or a negative error code.  The shapes are the
 * generator's (the paper's Tier-2 kernel of Sec. III-C re-derived per
 * class); the index into this list names a shape below. */
int eri_class_shapes(int la, int lb, int lc, int ld, int32_t* info, int max);

/* Preferred cooperative shape and vote form of a class for one kind of
 * contraction: kind 0 deep (more than 12 primitive quartets per part), 1
 * shallow (2 to 12), 2 single primitive quartet; shape = an index into
 * eri_class_shapes (-1 clears the entry); votes 0 (the class table of
 * eri_set_class_votes, else the static rule), 1 predicated, 2 warp votes.
 * Written by the autotuner; applies to plans with default generator options
 * built afterwards, process-wide.  An index beyond the class's list is
 * ignored at plan time. */
int eri_set_class_shape(int la, int lb, int lc, int ld, int kind, int shape, int votes);

/* Cooperative shape of launch i of a plan (see eri_plan_launch_info): info
 * (host, 4 int32) = {kind, shape index, team lanes T, vote form 1 or 2}, or
 * {-1, -1, 0, 0} for a launch of another tier.  ERI_EINVAL for a bad index. */
int eri_plan_launch_shape(const eri_plan_t* plan, int i, int32_t* info);

/* Capture eri_compute(plan, out, stream) into a CUDA graph held by the plan
 * (stream must not be the legacy default stream; launch timing is off in the
 * graph), and replay it with eri_plan_graph_launch: all of the plan's class
 * launches go out as one graph launch. */
int eri_plan_graph_capture(eri_plan_t* plan, double* out, void* stream);
/* The same for eri_compute_jk(plan, density, nbf, J, K, stream): each replay
 * adds into J and K (zero them between replays as needed).  The plan's block
 * buffer is allocated before the capture.  Errors as eri_compute_jk. */
int eri_plan_graph_capture_jk(eri_plan_t* plan, const double* density, int32_t nbf, double* J, double* K,
                              void* stream);
int eri_plan_graph_launch(eri_plan_t* plan, void* stream);

/* Release the plan and its device memory.  A plan from eri_plan_on_stream
 * frees its memory stream-ordered on its stream and returns at once; any
 * other plan synchronises the device first. */
int eri_plan_destroy(eri_plan_t* plan);

/* Diagnostic: the device Boys function on its own.  F_m(T) = int_0^1
 * t^(2m) exp(-T t^2) dt (Sec. II-A, the base of Eq. 2) for m = 0..L, for each
 * of n arguments T[i] >= 0 (device memory), into F (device, [n][L + 1]),
 * asynchronously on stream.  form selects the routine of one tier: 0 the
 * compiled register-tier kernels' (compile-time order), 1 the
 * team-cooperative executor's, 2 the thread-per-quartet executor's.
 * Errors: ERI_EINVAL for L outside 0..16, a bad form or NULL pointers. */
int eri_boys_eval(const double* T, int64_t n, int32_t L, int32_t form, double* F, void* stream);

/* Message for the calling thread's last error ("" if none). */
const char* eri_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ERI_H */
