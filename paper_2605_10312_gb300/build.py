"""Build of the CUDA library: run the generator, compile for sm_103a, link.

Steps (FusionRCG Sec. IV, stages 8-9):
  1. class programs for every class (default options) -> eri_programs.bin,
     together with the Boys Taylor table and the transform coefficients;
  2. straight-line register-tier kernels for the classes whose program is
     small enough to compile quickly, one translation unit per class, and
     the registry that lists them;
  3. nvcc -gencode arch=compute_103a,code=sm_103a for every unit, in
     parallel, then one shared library liberi.so.
Every program is checked for in-bounds indexes (gen.verify) before it is
written.
Everything lands in paper_2605_10312_gb300/_build/.  Units whose source did
not change are not recompiled.
"""
from __future__ import annotations

import hashlib
import math
import multiprocessing as mp
import os
import re
import shutil
import struct
import subprocess
import sys
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(HERE, "_build")
GEN_DIR = os.path.join(BUILD, "gen")
LIB = os.path.join(BUILD, "liberi.so")
NVCC_ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + CSRC, "-I" + os.path.join(ROOT, "include")]
# straight-line size (VRR terms + 1.5 x Phase-2 operations) up to which a
# class gets a compiled register-tier kernel; larger classes run as programs
REG_TIER_MAX = 3000
# cooperative shapes shipped per class besides the generator's choices, for
# the autotuner to time (the next best by the generator's score)
COOP_ALTS = 2

# classes and option variants of the paper's ablations (Sec. V-B): axis rule,
# DSA off, materialize-then-transform, Cartesian output
ABLATION_CLASSES = [(1, 1, 1, 1), (2, 1, 2, 1), (2, 2, 2, 1), (2, 2, 2, 2), (3, 3, 2, 2), (3, 3, 3, 3)]
ABLATION_OPTS = [("common", "dsa", "stepwise"), ("literal", "dsa", "stepwise"), ("prose", "level", "stepwise"),
                 ("prose", "dsa", "materialize"), ("prose", "dsa", "cart")]

AXIS = {"prose": 0, "literal": 1, "common": 2}
SCHED = {"dsa": 0, "level": 1}
SPH = {"stepwise": 0, "materialize": 1, "cart": 2}


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def boys_table(ngrid=362, ncol=24, step=0.1, dps=32):
    """F_n(T_k), n < ncol, T_k = k step: F_n(T) = 1F1(n+1/2; n+3/2; -T)/(2n+1)
    evaluated in high precision (mpmath)."""
    import mpmath
    mpmath.mp.dps = dps
    out = np.zeros((ngrid, ncol))
    for k in range(ngrid):
        T = mpmath.mpf(k) * mpmath.mpf(step)
        for n in range(ncol):
            v = mpmath.hyp1f1(n + mpmath.mpf(1) / 2, n + mpmath.mpf(3) / 2, -T) / (2 * n + 1)
            out[k, n] = float(v)
    return out


def _class_job(args):
    ls, opts, want_reg = args[:3]
    force_coop = len(args) > 3 and args[3]
    sys.setrecursionlimit(100000)
    from paper_2605_10312_gb300.gen import emit_cuda, encode, program, verify
    prog = program.make(*ls, *opts)
    enc = encode.encode(prog)
    ncoef = len(encode.coef_table())
    # every index a program-driven kernel takes from a descriptor is in bounds
    verify.check(ls, verify.verify_encoded(enc, ncoef))
    c = prog.counts()
    rec = dict(ls=ls, opts=opts, nh=enc.nh, nslot=enc.nslot, L=enc.L, n1=int(enc.ph1.shape[0]),
               n2=int(enc.ph2.shape[0]), kmax=enc.kmax, dims=enc.out_dims, flops_prim=float(c["per_prim_flops"]),
               flops_p2=float(c["p2_flops"]), ph1=enc.ph1.tobytes(), ph2=enc.ph2.tobytes(),
               size=c["vrr_instr"] + 1.5 * c["p2_instr"], counts=c)
    if want_reg and rec["size"] <= REG_TIER_MAX:
        rec["cuda"] = emit_cuda.emit_class(prog, "reg")
        rec["kname"] = emit_cuda.kernel_name(ls, "reg")
        # the reduced-precision form (FP32 recurrences) of the same schedule
        rec["cuda_f32"] = emit_cuda.emit_class(prog, "reg", real="float")
        rec["kname_f32"] = emit_cuda.kernel_name(ls, "reg", real="float")
    if want_reg or force_coop:
        # team-cooperative form of every class (the tier of the classes too
        # large for straight-line code; for the others an alternative the
        # autotuner and the persistent launch can take)
        from paper_2605_10312_gb300.gen import coop

        def pack(cp):
            return dict(T=cp.T, ilp=cp.ilp, nh=cp.nh, nslot=cp.nslot, L=cp.L, dims=cp.out_dims,
                        steps1=cp.steps1.tobytes(), steps2=cp.steps2.tobytes(), nw1=int(cp.steps1.shape[0]),
                        nw2=int(cp.steps2.shape[0]), ph1=cp.ph1.tobytes(), ph2=cp.ph2.tobytes(),
                        n1=int(cp.ph1.shape[0]), n2=int(cp.ph2.shape[0]), eff1=cp.eff1, eff2=cp.eff2,
                        issue=coop.fp64_issue(cp), lag=cp.lag, steps=coop.shape_key(cp)[2:],
                        wf=coop.shared_wavefronts(cp, cp.nslot * 8 + coop.DEEP_ROWS * coop.ROW_BYTES + cp.nh * 8
                                                  <= 227 * 1024))
        if want_reg:
            deep, shallow, alts = coop.choose_both(prog, alts=COOP_ALTS)
        else:
            (deep, shallow), alts = coop.choose_both(prog), []
        for cp in [deep, shallow] + list(alts):
            if cp is not None:
                verify.check(ls, verify.verify_coop(cp, prog.L, ncoef))
        rec["coop"] = pack(deep)
        # a second shape for shallow contractions, when it differs
        if shallow is not None and coop.shape_key(shallow) != coop.shape_key(deep):
            rec["coop_shallow"] = pack(shallow)
        # other shapes the autotuner may time against these
        rec["coop_alts"] = [pack(cp) for cp in alts]
    return rec


def generate(classes, opts=("prose", "dsa", "stepwise"), want_reg=True, jobs=None, log=print, extra=()):
    t0 = time.time()
    jobs = jobs or max(1, os.cpu_count() or 1)
    work = [(tuple(ls), tuple(opts), want_reg) for ls in classes] + list(extra)
    # heaviest first so the pool ends evenly
    work.sort(key=lambda w: -sum(w[0]) * 100 - w[0][0])
    ctx = mp.get_context("spawn")
    with ctx.Pool(jobs) as pool:
        recs = pool.map(_class_job, work, chunksize=1)
    log("generated {} class programs in {:.1f}s".format(len(recs), time.time() - t0))
    return recs


def write_blob(path, recs, boys, c2s):
    with open(path + ".tmp", "wb") as f:
        f.write(b"ERIPRG03")
        f.write(struct.pack("<I", boys.size))
        f.write(np.ascontiguousarray(boys, dtype="<f8").tobytes())
        f.write(struct.pack("<I", len(c2s)))
        f.write(np.asarray(c2s, dtype="<f8").tobytes())
        f.write(struct.pack("<I", len(recs)))
        for r in recs:
            o = r["opts"]
            f.write(struct.pack("<8b", *r["ls"], AXIS[o[0]], SCHED[o[1]], SPH[o[2]], 1 if "cuda" in r else 0))
            f.write(struct.pack("<10i", r["nh"], r["nslot"], r["L"], r["n1"], r["n2"], r["kmax"], *r["dims"]))
            f.write(struct.pack("<2d", r["flops_prim"], r["flops_p2"]))
            f.write(r["ph1"])
            f.write(r["ph2"])
        # team-cooperative programs: the deep-contraction shape of every class,
        # then the shallow-contraction shapes that differ from it, then the
        # autotuner's alternative shapes (any number per class)
        for key in ("coop", "coop_shallow"):
            _write_coops(f, [(r, r[key]) for r in recs if key in r])
        _write_coops(f, [(r, c) for r in recs for c in r.get("coop_alts", ())])
    os.replace(path + ".tmp", path)


def _write_coops(f, coops):
    f.write(struct.pack("<I", len(coops)))
    for r, c in coops:
        o = r["opts"]
        f.write(struct.pack("<8b", *r["ls"], AXIS[o[0]], SCHED[o[1]], SPH[o[2]], c["ilp"]))
        f.write(struct.pack("<15i", c["T"], c["nh"], c["nslot"], c["L"], c["nw1"], c["nw2"], c["n1"], c["n2"],
                            *c["dims"], c["lag"], *c["steps"]))
        f.write(struct.pack("<2d", r["flops_prim"], r["flops_p2"]))
        f.write(c["steps1"])
        f.write(c["steps2"])
        f.write(c["ph1"])
        f.write(c["ph2"])


def _registry(knames):
    """Registry unit of the compiled register-tier kernels: the names
    eri_<la><lb><lc><ld>_reg (FP64) and ..._reg_f32 (FP32 recurrences)."""
    lines = ['#include "eri_common.cuh"', "struct EriRegEntry { int8_t ls[4]; const void* fn; };"]
    for table, suffix in (("eri_reg", "_reg"), ("eri_reg_f32", "_reg_f32")):
        regs = sorted(k for k in knames if k.endswith(suffix))
        for k in regs:
            lines.append('extern "C" __global__ void {}(const EriLaunchArgs a);'.format(k))
        lines.append('extern "C" const EriRegEntry {}_table[] = {{'.format(table))
        for k in regs:
            ls = k.split("_")[1]
            lines.append("  {{{{{}, {}, {}, {}}}, (const void*){}}},".format(*ls, k))
        lines.append("  {{0, 0, 0, 0}, nullptr}};")
        lines.append('extern "C" const int {}_count = {};'.format(table, len(regs)))
    return "\n".join(lines) + "\n"


# A register-tier kernel whose ptxas spill stores exceed this is left out of
# the registry: its class runs on the cooperative tier.  Measured: the FP64
# (fp|pp) kernel came out at 32 registers with 47 KB of spill stores (every
# other kernel of its size uses 255 registers and spills at most 13 KB).
REG_SPILL_MAX = 16 * 1024


def _spill_bytes(obj):
    """Spill stores ptxas reported for a unit (the largest of its functions),
    kept beside the object when it was compiled."""
    try:
        return int(open(obj + ".spill").read())
    except (OSError, ValueError):
        return 0


def _write_if_changed(path, text):
    if os.path.exists(path) and open(path).read() == text:
        return
    with open(path, "w") as f:
        f.write(text)


def _compile(src, obj, extra=()):
    key = hashlib.sha256()
    heads = [os.path.join(CSRC, "eri_common.cuh"), os.path.join(ROOT, "include", "eri.h")]
    # project headers the unit includes by name
    for name in re.findall(r'^#include "([^"]+)"', open(src).read(), flags=re.M):
        h = os.path.join(CSRC, name)
        if os.path.exists(h) and h not in heads:
            heads.append(h)
    for p in [src] + heads:
        key.update(open(p, "rb").read())
    report = os.path.basename(src).startswith("eri_") and "_reg" in os.path.basename(src)
    key.update(" ".join(NVCC_ARCH + NVCC_FLAGS + list(extra) + (["-Xptxas", "-v"] if report else [])).encode())
    stamp = obj + ".key"
    h = key.hexdigest()
    if os.path.exists(obj) and os.path.exists(stamp) and open(stamp).read() == h:
        return 0.0
    t = time.time()
    cmd = [_nvcc()] + NVCC_ARCH + NVCC_FLAGS + list(extra) + (["-Xptxas", "-v"] if report else []) + \
        ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for {}:\n{}".format(src, r.stderr[-4000:]))
    if report:
        spills = [int(x) for x in re.findall(r"(\d+) bytes spill stores", r.stderr)]
        open(obj + ".spill", "w").write(str(max(spills, default=0)))
    open(stamp, "w").write(h)
    return time.time() - t


def build(force=False, jobs=None, log=print):
    """Generate, compile and link liberi.so (and the fp_peak tool)."""
    from paper_2605_10312_gb300.gen import encode, program
    os.makedirs(GEN_DIR, exist_ok=True)
    jobs = jobs or max(1, os.cpu_count() or 1)
    t0 = time.time()
    gen_key = hashlib.sha256()
    for fn in sorted(os.listdir(os.path.join(HERE, "gen"))):
        if fn.endswith(".py"):
            gen_key.update(open(os.path.join(HERE, "gen", fn), "rb").read())
    gen_key.update(open(__file__, "rb").read())
    gen_key = gen_key.hexdigest()
    blob = os.path.join(BUILD, "eri_programs.bin")
    stamp = os.path.join(BUILD, "gen.key")
    if force or not (os.path.exists(blob) and os.path.exists(stamp) and open(stamp).read() == gen_key):
        # ablation variants (program and cooperative forms, no compiled kernel)
        extra = [(tuple(ls), tuple(o), False, True) for ls in ABLATION_CLASSES for o in ABLATION_OPTS]
        allrecs = generate(program.all_classes(), jobs=jobs, log=log, extra=extra)
        recs = [r for r in allrecs if tuple(r["opts"]) == ("prose", "dsa", "stepwise")]
        abl = [r for r in allrecs if tuple(r["opts"]) != ("prose", "dsa", "stepwise")]
        boys = boys_table()
        write_blob(blob, recs, boys, encode.coef_table())
        write_blob(os.path.join(BUILD, "eri_programs_ablation.bin"), abl, boys, encode.coef_table())
        for r in recs:
            if "cuda" in r:
                _write_if_changed(os.path.join(GEN_DIR, r["kname"] + ".cu"), r["cuda"])
            if "cuda_f32" in r:
                _write_if_changed(os.path.join(GEN_DIR, r["kname_f32"] + ".cu"), r["cuda_f32"])
        # class table for the docs and the benchmark: per-class counts
        with open(os.path.join(BUILD, "classes.tsv"), "w") as f:
            f.write("la\tlb\tlc\tld\ttier\tvrr_nodes\tpeak_live\tnslot\tnh\tnout\tper_prim_flops\tp2_flops"
                    "\tcoop_T\tcoop_ilp\tcoop_nslot\tcoop_eff1\tcoop_eff2\tshallow_T\tshallow_ilp"
                    "\tcoop_fp64_ceil1\tcoop_fp64_ceil2\tcoop_wave_steps1\tcoop_wave_steps2"
                    "\tcoop_smem_wf1\tcoop_smem_ideal1\tcoop_smem_wf2\tcoop_smem_ideal2\n")
            for r in sorted(recs, key=lambda r: r["ls"]):
                c = r["counts"]
                cp = r.get("coop")
                f.write("\t".join(str(x) for x in (*r["ls"], "reg" if "cuda" in r else "coop", c["vrr_nodes"],
                                                   c["peak_live"], r["nslot"], c["nh"], c["nout"],
                                                   c["per_prim_flops"], c["p2_flops"],
                                                   cp["T"] if cp else "", cp["ilp"] if cp else "",
                                                   cp["nslot"] if cp else "",
                                                   round(cp["eff1"], 3) if cp else "",
                                                   round(cp["eff2"], 3) if cp else "",
                                                   r["coop_shallow"]["T"] if "coop_shallow" in r else "",
                                                   r["coop_shallow"]["ilp"] if "coop_shallow" in r else "",
                                                   # FP64 issue ceilings of the deep shape: algorithmic
                                                   # flops / (64 x FP64 warp-instructions)
                                                   round(c["vrr_flops"] / (64 * max(1, cp["issue"][0])), 3) if cp else "",
                                                   round(c["p2_flops"] / (64 * max(1, cp["issue"][1])), 3)
                                                   if cp else "",
                                                   # steps per wave of each phase; modelled shared-memory
                                                   # wavefronts of the value slots and the conflict-free
                                                   # count (Phase 1 per primitive quartet, Phase 2 per
                                                   # shell quartet)
                                                   *(cp["steps"] if cp else ("", "")),
                                                   *(cp["wf"] if cp else ("", "", "", "")))) + "\n")
        open(stamp, "w").write(gen_key)
    units = [os.path.join(CSRC, "eri_runtime.cu"), os.path.join(CSRC, "eri_exec.cu"),
             os.path.join(CSRC, "eri_coop.cu"), os.path.join(CSRC, "eri_digest.cu"),
             os.path.join(CSRC, "eri_screen.cu")]
    units += sorted(os.path.join(GEN_DIR, f) for f in os.listdir(GEN_DIR)
                    if f.endswith("_reg.cu") or f.endswith("_reg_f32.cu"))
    units.sort(key=lambda u: -os.path.getsize(u))  # largest first: the pool ends evenly
    objs = [os.path.join(BUILD, os.path.basename(u)[:-3] + ".o") for u in units]
    # drop objects of classes no longer generated
    keep = set(objs)
    for f in os.listdir(BUILD):
        p = os.path.join(BUILD, f)
        if (f.endswith("_reg.o") or f.endswith("_reg_f32.o")) and p not in keep:
            os.remove(p)
    t1 = time.time()
    with ThreadPoolExecutor(jobs) as ex:
        times = list(ex.map(lambda so: _compile(*so), zip(units, objs)))
    # the registry of the register-tier kernels, less those that spill past
    # REG_SPILL_MAX (their classes fall to the cooperative tier)
    regs, dropped = [], []
    for u, o in zip(units, objs):
        name = os.path.basename(u)[:-3]
        if name.endswith("_reg") or name.endswith("_reg_f32"):
            (dropped if _spill_bytes(o) > REG_SPILL_MAX else regs).append(name)
    if dropped:
        log("register-tier kernels left out for spilling over {} B: {}".format(REG_SPILL_MAX, ", ".join(dropped)))
    reg_src = os.path.join(GEN_DIR, "eri_registry.cu")
    _write_if_changed(reg_src, _registry(regs))
    objs.append(os.path.join(BUILD, "eri_registry.o"))
    times.append(_compile(reg_src, objs[-1]))
    log("compiled {} units ({} rebuilt) in {:.1f}s".format(len(objs), sum(1 for t in times if t > 0),
                                                          time.time() - t1))
    cmd = [_nvcc()] + NVCC_ARCH + ["-shared", "-o", LIB + ".tmp"] + objs + ["-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr[-4000:])
    os.replace(LIB + ".tmp", LIB)
    peak_src = os.path.join(CSRC, "fp_peak.cu")
    peak_bin = os.path.join(BUILD, "fp_peak")
    if not os.path.exists(peak_bin) or os.path.getmtime(peak_bin) < os.path.getmtime(peak_src):
        subprocess.run([_nvcc()] + NVCC_ARCH + ["-O3", "-o", peak_bin, peak_src], check=True)
    log("built {} in {:.1f}s".format(LIB, time.time() - t0))
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv)
