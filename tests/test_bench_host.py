"""Host-side pieces of the benchmark's JSON line (no GPU): the class-mix
rate, canonical class labels, the workload config, the FP64 roofline
denominator and the oracle baseline's single-core leg."""
import numpy as np

import bench
from paper_2605_10312_gb300 import synth


def test_mix_rate_is_the_harmonic_mix_of_the_step():
    rates = {ls: 10.0 * (i + 1) for i, (ls, _) in enumerate(bench.SWEEP)}
    tot = sum(n for _, n in bench.SWEEP)
    t = sum(n / rates[ls] for ls, n in bench.SWEEP)
    assert abs(bench.mix_rate(rates) - tot / t) < 1e-9 * tot / t
    same = {ls: 7.0 for ls, _ in bench.SWEEP}
    assert abs(bench.mix_rate(same) - 7.0) < 1e-12


def test_class_labels_are_canonical():
    """Any shell order of a quartet maps to one label: pairs high l first,
    bra pair not below the ket pair."""
    b, q = synth.class_sweep((1, 3, 0, 2), 4, seed=5)
    perms = [(0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]
    for p in perms:
        inv, labels = bench._class_labels(b, q[:, list(p)])
        assert labels == ["fpds"] and (inv == 0).all()


def test_config_and_peak():
    c = bench.config_dict()
    assert c["quartets_per_step"] == sum(n for _, n in bench.SWEEP) == 2_200_000
    assert c["K_per_shell"] == [1, 3, 6] and c["box_angstrom"] == 10.0 and c["output"] == "spherical"
    assert "flushed" in c["l2"]
    # 1.683 FMA lanes per SM per clock x 2 flops x 152 SMs x 2070 MHz
    assert abs(bench.fp64_peak_tflops() - 1.683 * 2 * 152 * 2070e6 / 1e12) < 1e-9


def test_single_core_oracle_leg():
    parts = [((1, 1, 1, 1), *synth.class_sweep((1, 1, 1, 1), 64, kset=(1, 3), seed=1))]
    old = bench.SWEEP
    try:
        bench.SWEEP = [((1, 1, 1, 1), 64)]
        r = bench.single_core_baseline(parts, budget_s=0.2)
    finally:
        bench.SWEEP = old
    assert r["cores"] == 1 and r["value"] > 0 and r["per_class"]["pppp"] == r["value"]
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()
