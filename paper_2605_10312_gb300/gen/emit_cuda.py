"""Straight-line sm_103a CUDA for a class program (FusionRCG Sec. IV, stages
7-8: the accumulate-then-transform loop structure and kernel emission).

One thread evaluates one shell quartet (Algorithm 2): the two primitive-pair
loops enclose the set-up, the Boys function and the Phase-1 graph in its
schedule order, each target folded into its contracted accumulator; Phase 2
runs once after the loops and the block is stored through the quartet's
output strides.

Tiers (where Phase-1 intermediates live):
  "reg"    every value a local; the compiler keeps what fits in registers;
  "smem"   Phase-1 values in shared-memory slots from the lifetime
           allocator, [slot][thread] so that a warp's accesses are
           bank-conflict free; accumulators stay local;
  "global" Phase-1 values and accumulators in a coalesced global scratch,
           [slot][thread] across the whole grid (the paper's interleaved
           Tier-2 buffer).
"""
from __future__ import annotations

import numpy as np

from . import vrr

TIERS = ("reg", "smem", "global")
AX = "xyz"


def kernel_name(ls, tier, opts=None, real="double"):
    base = "eri_{}{}{}{}_{}".format(*ls, tier)
    if opts is not None and opts.key() != ("prose", "dsa", "stepwise"):
        base += "_" + "_".join(opts.key())
    if real == "float":
        base += "_f32"
    return base


def _coef_expr(sym, real="double"):
    kind, k = sym
    if real == "float":
        return "f{}_{}".format(kind, k) if kind in ("PA", "QC", "WP", "WQ") else "{}_{}".format(kind, k)
    if kind == "PA":
        return "bp.PA[{}]".format(k)
    if kind == "QC":
        return "kp.PA[{}]".format(k)
    if kind == "WP":
        return "pq.WP[{}]".format(k)
    if kind == "WQ":
        return "pq.WQ[{}]".format(k)
    return "{}_{}".format(kind, k)


def _coef_defs(syms, real="double"):
    """Definitions of the integer-multiple coefficients a class uses:
    c1z_k = k/(2 zeta), c2z_k = -k rho/(2 zeta^2), likewise for eta, and
    c3_k = k/(2(zeta+eta)).  In single precision every coefficient is
    formed in FP32 from the FP32 pair and primitive-quartet data."""
    lines = []
    if real == "float":
        src = {"PA": "bp.PA[{}]", "QC": "kp.PA[{}]", "WP": "pq.WP[{}]", "WQ": "pq.WQ[{}]"}
        for kind, k in sorted(s for s in syms if s[0] in src):
            lines.append("    const float f{}_{} = {};".format(kind, k, src[kind].format(k)))
        base = {"c1z": "bp.inv2z", "c1e": "kp.inv2z", "c2z": "(-bp.inv2z * pq.te)",
                "c2e": "(-kp.inv2z * pq.tz)", "c3": "(0.5f * pq.s)"}
        for kind, k in sorted(s for s in syms if s[0] in base):
            lines.append("    const float {}_{} = {}.0f * {};".format(kind, k, k, base[kind]))
        return lines
    need = sorted(s for s in syms if s[0] in ("c1z", "c2z", "c1e", "c2e", "c3"))
    have = set()

    def base(kind):
        if kind == "c1z":
            return "bp.inv2z"
        if kind == "c1e":
            return "kp.inv2z"
        if kind == "c2z":
            return "(-bp.inv2z * pq.te)"
        if kind == "c2e":
            return "(-kp.inv2z * pq.tz)"
        return "(0.5 * pq.s)"

    for kind, k in need:
        if (kind, 1) not in have:
            lines.append("    const double {}_1 = {};".format(kind, base(kind)))
            have.add((kind, 1))
        if k != 1:
            lines.append("    const double {0}_{1} = {1}.0 * {0}_1;".format(kind, k))
            have.add((kind, k))
    return lines


def _fmt(c, real="double"):
    r = repr(float(c))
    r = r if ("e" in r or "." in r) else r + ".0"
    return r + "f" if real == "float" else r


def emit_class(prog, tier="reg", threads=128, real="double"):
    """CUDA source of one class kernel.  real="float" (register tier only)
    gives the reduced-precision form: pair and quartet set-up, the Boys
    function and the output store in FP64, the recurrences, the
    contraction sums, HRR and the transform in FP32."""
    assert real == "double" or tier == "reg"
    R = real
    FMA = "fmaf" if real == "float" else "fma"
    ZERO = "0.0f" if real == "float" else "0.0"
    g = prog.g
    la, lb, lc, ld = prog.ls
    L = prog.L
    name = kernel_name(prog.ls, tier, prog.opts, real)
    nh = prog.nh
    out = []
    w = out.append
    c = prog.counts()
    w("// class ({} {} | {} {}), tier {}, axis rule {}, schedule {}, sph {}, recurrences in {}".format(
        la, lb, lc, ld, tier, *prog.opts.key(), R))
    w("// VRR nodes {}  PeakLive {}  slots {}  accumulators {}  outputs {}".format(
        c["vrr_nodes"], c["peak_live"], c["nslot"], c["nh"], c["nout"]))
    w("// flops per primitive quartet {}  Phase-2 flops {}".format(c["per_prim_flops"], c["p2_flops"]))
    w('#include "eri_common.cuh"')
    w("")
    if tier == "smem":
        w("extern __shared__ double eri_smem[];")
    w('extern "C" __global__ void __launch_bounds__({}) {}(const EriLaunchArgs a) {{'.format(threads, name))
    w("  // a.group lanes share one shell quartet and split its primitive quartets")
    w("  const int t = blockIdx.x * blockDim.x + threadIdx.x;")
    w("  const int G = a.group;")
    w("  const int qi = t / G, r = t - qi * G;")
    w("  const bool valid = qi < a.nq;")
    w("  const EriQuartetRec qr = a.quartets[valid ? qi : 0];")
    w("  const EriPairRec bra = a.pairs[ERI_PAIR_INDEX(qr.bra)];")
    w("  const EriPairRec ket = a.pairs[qr.ket];")
    w("  const bool acc = ERI_ACCUMULATE(qr.bra);")
    w("  const bool red = ERI_REDUCE(qr.bra);")
    if tier == "smem":
        w("  double* const S = eri_smem + threadIdx.x;")
        w("#define SV(i) S[(i) * {}]".format(threads))
    elif tier == "global":
        w("  double* const S = a.scratch + (int64_t)t;")
        w("#define SV(i) S[(int64_t)(i) * a.scratch_stride]")
    # accumulators
    if tier == "global":
        hbase = prog.nslot
        w("#define HV(i) S[(int64_t)({} + (i)) * a.scratch_stride]".format(hbase))
        w("  for (int i = 0; i < {}; ++i) HV(i) = 0.0;".format(nh))
        hname = lambda i: "HV({})".format(i)
    else:
        for i0 in range(0, nh, 16):
            w("  {} ".format(R) + ", ".join("h{} = {}".format(i, ZERO) for i in range(i0, min(nh, i0 + 16))) + ";")
        hname = lambda i: "h{}".format(i)
    w("  const int kk = ket.nprim;")
    w("  const int nk = valid ? bra.nprim : 0;")
    w("  int i = r / kk, j = r - (r / kk) * kk;")
    w("  while (i < nk) {")
    if real == "float":
        # FP32 set-up from the FP32 pair data; the Boys function in FP64
        w("    const EriPairPrimF bp = a.pprims_f[bra.prim_off + i];")
        w("    const EriPairPrimF kp = a.pprims_f[ket.prim_off + j];")
    else:
        w("    const EriPairPrim bp = a.pprims[bra.prim_off + i];")
        w("    const EriPairPrim kp = a.pprims[ket.prim_off + j];")
    w("    j += G;")
    w("    while (j >= kk) { j -= kk; ++i; }")
    if real == "float":
        w("    EriPrimQuartetF pq;")
        w("    eri_prim_quartet_f32(bp, kp, pq);")
        w("    double F[{}];".format(L + 1))
        w("    eri_boys<{}>((double)pq.T, F, a.boys_tab);".format(L))
        used_m = sorted(set(g.keys[v][2] for v in prog.order if not g.terms[v]))
        for m in used_m:
            w("    const float fF{0} = pq.pref * (float)F[{0}];".format(m))
    else:
        w("    EriPrimQuartet pq;")
        w("    eri_prim_quartet(bp, kp, pq);")
        w("    double F[{}];".format(L + 1))
        w("    eri_boys<{}>(pq.T, F, a.boys_tab);".format(L))
    for ln in _coef_defs(prog.coef_syms, real):
        w(ln)
    slot = prog.slot
    consumed = set(p for ts in g.terms for _, p in ts)

    def loc(v):
        return "v{}".format(v) if tier == "reg" else "SV({})".format(slot[v])

    for v in prog.order:
        ts = g.terms[v]
        tgt = g.target.get(v)
        if tier == "reg":
            ops = [(_coef_expr(cs, real), loc(p)) for cs, p in ts]
        else:
            ops = [(_coef_expr(cs), "r{}".format(k)) for k, (cs, p) in enumerate(ts)]
        if not ts:
            if real == "float":
                ops = [(None, "fF{}".format(g.keys[v][2]))]
            else:
                ops = [("pq.pref", "F[{}]".format(g.keys[v][2]))]
        fold = tgt is not None and v not in consumed and tier != "global"
        expr = hname(tgt) if fold else None
        for cexp, pv_ in ops:
            if cexp is None:
                expr = pv_ if expr is None else "{} + {}".format(expr, pv_)
            else:
                expr = "{} * {}".format(cexp, pv_) if expr is None else "{}({}, {}, {})".format(FMA, cexp, pv_, expr)
        loads = ""
        if tier != "reg" and ts:
            loads = " ".join("const double r{} = {};".format(k, loc(p)) for k, (cs, p) in enumerate(ts)) + " "
        if fold:
            line = "{}{} = {};".format(loads, hname(tgt), expr)
        elif tgt is not None:
            line = "{}const double x{} = {}; {} += x{};".format(loads, v, expr, hname(tgt), v)
            if v in consumed:
                line += " {} = x{};".format(loc(v), v) if tier != "reg" else ""
                if tier == "reg":
                    line = "{}const {} v{} = {}; {} += v{};".format(loads, R, v, expr, hname(tgt), v)
        else:
            line = "{}{}{} = {};".format(loads, "const {} ".format(R) if tier == "reg" else "", loc(v), expr)
        w("    " + ("{ " + line + " }" if tier != "reg" else line))
    w("  }")
    if tier != "global":
        # group reduction of the accumulators: reduce-scatter (each round
        # halves the vector a lane keeps, so a lane adds about nh values in
        # all) then all-gather back, instead of nh * log2(G) butterfly adds
        w("  if (G > 1) {")
        w("    const unsigned m = eri_group_mask(G);")
        w("    const int lane = threadIdx.x & 31;")
        names = [hname(i) for i in range(nh)]
        w("    int off = G >> 1;")
        # reduce-scatter rounds, vector halves stay in the low names
        vec = list(names)
        rounds = []
        for _ in range(5):
            rounds.append(list(vec))
            n = len(vec)
            half = n // 2
            w("    if (off > 0) {")
            w("      const bool up = (lane & off) != 0;")
            for i in range(half):
                lo, hi = vec[i], vec[half + i]
                w("      {{ const {2} snd = up ? {0} : {1}; const {2} kp = up ? {1} : {0}; "
                  "{0} = kp + __shfl_xor_sync(m, snd, off); }}".format(lo, hi, R))
            if n % 2:
                x = vec[n - 1]
                w("      {0} += __shfl_xor_sync(m, {0}, off);".format(x))
            w("      off >>= 1;")
            w("    }")
            vec = vec[:half] + ([vec[n - 1]] if n % 2 else [])
        # all-gather: undo the reduce-scatter rounds, last first; round k
        # used offset G >> (k + 1)
        for k in range(4, -1, -1):
            v = rounds[k]
            n = len(v)
            half = n // 2
            w("    if ((G >> {0}) > 0) {{".format(k + 1))
            w("      const int o2 = G >> {};".format(k + 1))
            w("      const bool up = (lane & o2) != 0;")
            for i in range(half):
                lo, hi = v[i], v[half + i]
                w("      {{ const {2} mine = {0}; const {2} oth = __shfl_xor_sync(m, mine, o2); "
                  "{0} = up ? oth : mine; {1} = up ? mine : oth; }}".format(lo, hi, R))
            w("    }")
        w("  }")
    w("  if (!valid || r != 0) return;")
    # Phase 2
    p2 = prog.p2

    def pv(i):
        return hname(i) if i < nh else "p{}".format(i)

    if real == "float":
        for i in range(3):
            w("  const float fAB{0} = (float)bra.AB[{0}], fCD{0} = (float)ket.AB[{0}];".format(i))
    for op in p2.ops:
        if op[0] == "hrr":
            _, d, hi, (sym, i), lo = op
            if real == "float":
                src = "fAB{}".format(i) if sym == "AB" else "fCD{}".format(i)
            else:
                src = "bra.AB[{}]".format(i) if sym == "AB" else "ket.AB[{}]".format(i)
            w("  const {} p{} = {}({}, {}, {});".format(R, d, FMA, src, pv(lo), pv(hi)))
        else:
            _, d, terms = op
            expr = "{} * {}".format(_fmt(terms[0][0], real), pv(terms[0][1]))
            for cc, s in terms[1:]:
                expr = "{}({}, {}, {})".format(FMA, _fmt(cc, real), pv(s), expr)
            w("  const {} p{} = {};".format(R, d, expr))
    w("  double* const o = a.out + qr.out_off;")
    dims = p2.out_dims
    for k, vid in enumerate(p2.outputs):
        idx = np.unravel_index(k, dims)
        terms = []
        for axis, ii in enumerate(idx):
            if ii:
                terms.append("{}*qr.st[{}]".format(int(ii), axis))
        off = " + ".join(terms) if terms else "0"
        w("  eri_st(o + {}, {}{}, acc, red);".format(off, "(double)" if real == "float" else "", pv(vid)))
    if tier in ("smem", "global"):
        w("#undef SV")
    if tier == "global":
        w("#undef HV")
    w("}")
    return "\n".join(out) + "\n"


