"""Host-side checks of the code generator (FusionRCG Sec. III-A, III-B, IV):
graph construction under each axis rule, DSA scheduling, PeakLive, the
lifetime slot allocator, the Phase-2 graph in every transform mode, and the
encoded programs -- evaluated on the CPU against the oracle."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2605_10312_gb300 import synth
from paper_2605_10312_gb300.gen import cart, coop, encode, hrr, program, sph, vrr
from gen_eval import evaluate, run_coop, run_encoded
from ref import blocks, within


def test_cartesian_order():
    assert cart.tuples(2) == ((2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2))
    for l in range(9):
        assert [cart.index(t) for t in cart.tuples(l)] == list(range(cart.ncart(l)))


def test_generator_sph_matches_oracle():
    # two independent derivations: solid-harmonic recurrence vs closed form
    for l in range(5):
        np.testing.assert_allclose(sph.matrix(l), oracle.cart2sph(l), atol=2e-15)


@pytest.mark.parametrize("rule", vrr.AXIS_RULES)
@pytest.mark.parametrize("ls", [(1, 1, 1, 1), (2, 2, 1, 1), (2, 1, 2, 2), (3, 0, 1, 2)])
def test_vrr_graph_is_complete_and_acyclic(rule, ls):
    g = vrr.build(*ls, rule=rule)
    E, F = vrr.h_layout(*ls)
    assert sorted(g.target.values()) == list(range(len(E) * len(F)))
    for v, ts in enumerate(g.terms):
        e, f, m = g.keys[v]
        assert m <= sum(ls) - sum(e) - sum(f)
        for _, p in ts:
            assert p < v  # parents are created first
        if not ts:
            assert e == (0, 0, 0) and f == (0, 0, 0)


def test_node_counts_by_axis_rule():
    # (2,2,1,1): consumer-first 521, Algorithm 1 as printed 718, bra-first 671
    got = {r: len(vrr.build(2, 2, 1, 1, r)) for r in vrr.AXIS_RULES}
    assert got == {"prose": 521, "literal": 718, "common": 671}
    assert len(vrr.build(1, 1, 1, 1)) == 146
    assert len(vrr.build(2, 2, 2, 2)) == 2330


@pytest.mark.parametrize("how", vrr.SCHEDULES)
@pytest.mark.parametrize("ls", [(1, 1, 1, 1), (2, 2, 1, 1), (2, 2, 2, 2)])
def test_schedule_and_slots(how, ls):
    g = vrr.build(*ls)
    order = vrr.schedule(g, how)
    assert vrr.check_topological(g, order)
    peak = vrr.peak_live(g, order)
    slot, nslot = vrr.allocate_slots(g, order)
    assert vrr.verify_slots(g, order, slot)
    assert nslot <= peak


def test_dsa_lowers_peak_live():
    for ls in [(1, 1, 1, 1), (2, 2, 1, 1), (2, 2, 2, 2)]:
        g = vrr.build(*ls)
        assert vrr.peak_live(g, vrr.schedule(g, "dsa")) < vrr.peak_live(g, vrr.schedule(g, "level"))


def test_dsa_score_by_brute_force():
    """Eq. 7 scores against a direct set computation of Reach(v)."""
    g = vrr.build(1, 1, 1, 0)
    cons = [[] for _ in range(len(g))]
    for v, ts in enumerate(g.terms):
        for _, p in ts:
            cons[p].append(v)
    outd = [len(set(c)) for c in cons]
    ind = [len(set(p for _, p in ts)) for ts in g.terms]
    s = vrr.dsa_scores(g, window=64)
    for v in range(len(g)):
        reach, stack = set(), [v]
        while stack:
            w = stack.pop()
            if w not in reach:
                reach.add(w)
                stack.extend(cons[w])
        assert s[v] == sum(outd[w] - ind[w] for w in reach)


def test_stepwise_saves_operations():
    # Eq. 16 vs Eq. 17: the stepwise order needs fewer operations at high l
    for ls in [(2, 2, 2, 2), (4, 4, 4, 4)]:
        st = hrr.op_counts(hrr.build(*ls, "stepwise"))[0]
        ma = hrr.op_counts(hrr.build(*ls, "materialize"))[0]
        assert st < ma


OPTS = [("prose", "dsa", "stepwise"), ("literal", "level", "materialize"), ("common", "dsa", "cart"),
        ("prose", "level", "stepwise")]


@pytest.mark.parametrize("opts", OPTS)
@pytest.mark.parametrize("ls", [(0, 0, 0, 0), (1, 0, 0, 0), (1, 1, 1, 1), (2, 1, 0, 1), (0, 2, 1, 2), (3, 1, 2, 0),
                                (2, 2, 2, 1)])
def test_program_matches_oracle(ls, opts):
    """The graph program (interpreted in numpy) and its encoded descriptor
    stream both reproduce the oracle."""
    prog = program.make(*ls, *opts)
    basis, q = synth.class_sweep(ls, 3, kset=(1, 2), seed=9, box_angstrom=3.0, exp_range=(0.1, 30))
    ref, off = blocks(basis, q, cart=(opts[2] == "cart"))
    ref = ref.reshape(q.shape[0], -1)
    a = evaluate(prog, basis, q)
    b = run_encoded(encode.encode(prog), prog, basis, q)
    assert within(a, ref).all()
    assert within(b, ref).all()


def test_all_classes_enumerated():
    cls = program.all_classes()
    assert len(cls) == 325 and len(set(cls)) == 325
    # every ordered combination maps to one class by bra-ket exchange
    for ls in itertools.product(range(5), repeat=4):
        a, b = (ls[0], ls[1]), (ls[2], ls[3])
        key = a + b if program.pair_rank(*a) >= program.pair_rank(*b) else b + a
        assert key in cls


@pytest.mark.parametrize("T,ilp", [(32, 2), (64, 2), (128, 2), (128, 4)])
@pytest.mark.parametrize("ls", [(1, 1, 1, 1), (0, 2, 1, 2), (2, 2, 2, 1), (4, 0, 2, 1), (3, 3, 1, 0)])
def test_coop_program_matches_oracle(ls, T, ilp):
    """Team-cooperative waves (bounded-width DSA list schedule, slots reused
    only across waves) reproduce the oracle, wave semantics included."""
    prog = program.make(*ls)
    cp = coop.build(prog, T, ilp)
    assert (int(cp.steps1.sum()) + coop.PREFETCH_STEPS) * T * ilp == cp.ph1.shape[0]
    basis, q = synth.class_sweep(ls, 3, kset=(1, 2), seed=13, box_angstrom=3.0, exp_range=(0.1, 30))
    ref, _ = blocks(basis, q)
    got = run_coop(cp, prog, basis, q)
    assert within(got, ref.reshape(q.shape[0], -1)).all()


@pytest.mark.parametrize("T,ilp,k", [(32, 2, 4), (64, 2, 2), (32, 4, 3)])
@pytest.mark.parametrize("ls", [(2, 2, 1, 1), (3, 1, 2, 0)])
def test_coop_multistep_waves_match_oracle(ls, T, ilp, k):
    """Waves of several steps (no barrier between the steps of a wave) keep
    the program exact: nodes of a wave are independent and a slot is reused
    only after the wave of its last reader."""
    prog = program.make(*ls)
    cp = coop.build(prog, T, ilp, k)
    assert int(cp.steps1.max()) > 1
    assert (int(cp.steps1.sum()) + coop.PREFETCH_STEPS) * T * ilp == cp.ph1.shape[0]
    basis, q = synth.class_sweep(ls, 3, kset=(1, 2), seed=17, box_angstrom=3.0, exp_range=(0.1, 30))
    ref, _ = blocks(basis, q)
    got = run_coop(cp, prog, basis, q)
    assert within(got, ref.reshape(q.shape[0], -1)).all()


@pytest.mark.parametrize("T,ilp,k2", [(32, 2, 8), (64, 2, 2), (128, 2, 4)])
@pytest.mark.parametrize("ls", [(2, 2, 1, 1), (3, 2, 2, 1)])
def test_coop_wider_phase2_waves_match_oracle(ls, T, ilp, k2):
    """Phase-2 waves of several steps over one-step Phase-1 waves (the two
    phases are scheduled and allocated apart; Phase 2 reads H and its own
    slots) reproduce the oracle, and the verifier accepts the program."""
    from paper_2605_10312_gb300.gen import verify
    prog = program.make(*ls)
    cp = coop.build(prog, T, ilp, 1, wave_steps2=k2)
    assert int(cp.steps1.max()) == 1 and int(cp.steps2.max()) > 1
    assert len(cp.steps2) < len(coop.build(prog, T, ilp, 1).steps2)
    assert verify.verify_coop(cp, prog.L, len(encode.coef_table())) == []
    basis, q = synth.class_sweep(ls, 3, kset=(1, 2), seed=23, box_angstrom=3.0, exp_range=(0.1, 30))
    ref, _ = blocks(basis, q)
    got = run_coop(cp, prog, basis, q)
    assert within(got, ref.reshape(q.shape[0], -1)).all()


@pytest.mark.parametrize("ls", [(2, 2, 1, 1), (3, 1, 2, 0)])
def test_coop_512_lane_program_matches_oracle(ls):
    """The widest team (512 lanes, two nodes per lane, waves of up to two
    steps of 1024 nodes) is the same program form: every wave fits in a few
    lane slots of one step, most lanes are no-ops, and the result is exact."""
    prog = program.make(*ls)
    cp = coop.build(prog, *coop.WIDEST_SHAPE, 2)
    assert cp.T * cp.ilp * 2 <= coop.WAVE_NODES_MAX
    assert (int(cp.steps1.sum()) + coop.PREFETCH_STEPS) * cp.T * cp.ilp == cp.ph1.shape[0]
    basis, q = synth.class_sweep(ls, 3, kset=(1, 2), seed=19, box_angstrom=3.0, exp_range=(0.1, 30))
    ref, _ = blocks(basis, q)
    got = run_coop(cp, prog, basis, q)
    assert within(got, ref.reshape(q.shape[0], -1)).all()


class _FakeProg:
    """Stands in for a class program in the shape-selection test: a live
    set of `slots` values at a 64-node wave, growing with the wave width."""

    def __init__(self, slots, nh):
        self.slots, self.nh = slots, nh


def test_widest_team_only_where_a_256_lane_team_is_alone(monkeypatch):
    """choose_both builds the 512-lane shape only when a 256-lane team holds
    its SM alone even with H in global memory (the runtime then keeps eight
    warps per SM; the wider team keeps sixteen).  Where two 256-lane teams
    fit, the wider team would only lose lane efficiency."""
    built = []

    def fake_build(prog, T, ilp, k=1, lag=1, wave_steps2=None, **kw):
        built.append((T, ilp, k))
        width = T * ilp * k
        nslot = prog.slots + width
        eff = 0.98 - 0.00015 * width
        z = np.zeros((1, 4), dtype=np.uint32)
        s = np.ones(1, dtype=np.uint32)
        return coop.CoopProgram(T, ilp, z, s, z, s, prog.nh, nslot, 16, (9, 9, 9, 9), eff, eff)

    monkeypatch.setattr(coop, "build", fake_build)
    # (gg|gg)-sized live set: a 256-lane team is alone even without H
    deep, shallow = coop.choose_both(_FakeProg(21000, 21025))
    assert coop.WIDEST_SHAPE + (1,) in built
    assert (deep.T, deep.ilp) == coop.WIDEST_SHAPE
    # its waves hold at most WAVE_NODES_MAX nodes: four steps
    assert coop.WIDEST_SHAPE + (4,) in built
    # a live set two 256-lane teams can share (H in global memory): no 512
    built.clear()
    deep, shallow = coop.choose_both(_FakeProg(11000, 12000))
    assert all(T < 512 for T, _, _ in built)
    assert deep.T < 512 and shallow.T < 512


def test_wave_schedule_respects_dependencies_and_width():
    g = vrr.build(2, 2, 2, 1)
    order = vrr.schedule(g)
    pos = np.empty(len(g), dtype=np.int64)
    pos[np.array(order)] = np.arange(len(g))
    par = [[p for _, p in ts] for ts in g.terms]
    waves = coop.wave_schedule(par, pos, 32)
    wave_of = {}
    for w, vs in enumerate(waves):
        assert 0 < len(vs) <= 32
        for v in vs:
            wave_of[v] = w
    for v, ps in enumerate(par):
        for p in ps:
            assert wave_of[p] < wave_of[v]
    slot, n = coop.allocate_over_waves(par, waves, np.ones(len(g), dtype=bool))
    # a slot is never shared by two values whose wave lifetimes overlap
    last = {v: max([wave_of[c] for c, ps in enumerate(par) if v in ps], default=wave_of[v]) for v in range(len(g))}
    owners = {}
    for v in sorted(range(len(g)), key=lambda v: wave_of[v]):
        s = int(slot[v])
        if s in owners:
            assert last[owners[s]] < wave_of[v]
        owners[s] = v


def test_coop_shallow_shape_prefers_narrow_teams():
    """With 12 coefficient rows instead of 32 a team needs less shared
    memory, so a mid-size class fits 16 one-warp teams per SM and takes the
    narrower (better-filled) waves; both choices are valid programs."""
    prog = program.make(1, 2, 1, 2)
    deep, shallow = coop.choose_both(prog)
    assert deep is not None and shallow is not None
    assert shallow.T < deep.T
    assert coop._score(shallow, coop.SHALLOW_ROWS) >= coop._score(deep, coop.SHALLOW_ROWS)
    assert coop._score(deep, coop.DEEP_ROWS) >= coop._score(shallow, coop.DEEP_ROWS)


@pytest.mark.parametrize("ls", [(1, 1, 1, 1), (2, 2, 1, 1), (3, 1, 2, 0), (2, 2, 2, 2), (4, 0, 2, 1)])
def test_generated_programs_are_in_bounds(ls):
    """Every index a program-driven kernel takes from a descriptor (slots,
    accumulators, coefficient-row entries, transform-table entries, output
    elements) lies in the region the kernel addresses with it."""
    from paper_2605_10312_gb300.gen import verify
    prog = program.make(*ls)
    ncoef = len(encode.coef_table())
    assert verify.verify_encoded(encode.encode(prog), ncoef) == []
    for T, ilp, k in ((32, 2, 1), (128, 4, 1), (64, 2, 2), (512, 2, 2)):
        assert verify.verify_coop(coop.build(prog, T, ilp, k), prog.L, ncoef) == []


def test_bounds_verifier_catches_planted_errors():
    """Out-of-range indexes planted in copies of a valid program (on the
    host) are each reported."""
    import copy
    from paper_2605_10312_gb300.gen import verify
    prog = program.make(2, 2, 1, 1)
    ncoef = len(encode.coef_table())
    cp = coop.build(prog, 32, 2)
    live1 = np.flatnonzero(((cp.ph1[:, 3] >> 16) & 0xC000) == 0)   # nodes with operands
    stores = np.flatnonzero((cp.ph2[:, 0] & 3) == 2)
    lins = np.flatnonzero((cp.ph2[:, 0] & 3) == 1)

    def planted(fn):
        c = copy.deepcopy(cp)
        fn(c)
        return verify.verify_coop(c, prog.L, ncoef)

    def operand(c):
        c.ph1[live1[0], 1] = (c.ph1[live1[0], 1] & 0xFFFF0000) | c.nslot
    def accumulator(c):
        c.ph1[live1[0], 0] = (c.ph1[live1[0], 0] & 0xFFFF) | ((c.nh + 1) << 16)
    def element(c):
        c.ph2[stores[0], 1] = np.prod(c.out_dims)
    def coefficient(c):
        c.ph2[lins[0], 3] = (c.ph2[lins[0], 3] & 0xFFFFFF00) | ncoef
    def prefetch(c):
        c.ph1[-1] = c.ph1[live1[0]]

    def orphan(c):
        # drop one target: its accumulator then has no owner
        t = np.flatnonzero((((c.ph1[:, 3] >> 16) & 0x8000) == 0) & ((c.ph1[:, 0] >> 16) > 0))[0]
        c.ph1[t, 0] = c.ph1[t, 0] & 0xFFFF
    for fn in (operand, accumulator, element, coefficient, prefetch, orphan):
        assert planted(fn), fn.__name__
    enc = encode.encode(prog)
    term = int(np.flatnonzero(((enc.ph1[:, 3] >> 16) & 3) != 2)[0])   # first node with operands
    bad = copy.deepcopy(enc)
    bad.ph1[term, 1] = enc.nslot
    assert verify.verify_encoded(bad, ncoef)


def test_fp64_issue_count_bounds():
    """The FP64 warp-instruction count of a cooperative program lies between
    the lane instructions packed 32 to a warp and one full warp-instruction
    set per occupied descriptor slot; the ceiling it gives is below 1."""
    prog = program.make(2, 2, 2, 1)
    c = prog.counts()
    cp = coop.build(prog, 64, 2)
    i1, i2 = coop.fp64_issue(cp)
    g = prog.g
    lane1 = sum(len(ts) for ts in g.terms)        # one instruction per term
    assert lane1 / 32 <= i1 <= 5 * int(cp.steps1.sum()) * (cp.T // 32) * cp.ilp
    ins2, _ = hrr.op_counts(prog.p2)
    assert ins2 / 32 <= i2
    assert c["vrr_flops"] / (64 * i1) < 1 and c["p2_flops"] / (64 * i2) < 1


def test_fp64_balance_over_sub_partitions():
    """The sub-partition balance of a wave lies in (0, 1]; a team whose
    FP64 work sits on one warp of four scores 1/4; the shipped (ff|ff) program
    (128-lane teams, one warp per sub-partition) balances its waves to better
    than 0.8."""
    import copy
    prog = program.make(3, 3, 3, 3)
    deep, _ = coop.choose_both(prog)
    assert deep.T == 128
    b = coop.fp64_balance(deep)
    assert 0.8 < b <= 1.0
    # every descriptor of warps 1-3 made a no-op: all work on sub-partition 0
    one = copy.deepcopy(deep)
    W = one.T * one.ilp
    n = int(one.steps1.sum())
    ph = one.ph1[: n * W].reshape(n, one.T, one.ilp, 4)
    ph[:, 32:] = 0
    ph[:, 32:, :, 3] = 0x8000 << 16
    assert abs(coop.fp64_balance(one) - 0.25) < 1e-12


def test_gggg_production_program_matches_oracle():
    """The (gg|gg) cooperative program the build ships (512-lane teams,
    waves of up to four steps), walked wave by wave on the CPU, reproduces the
    oracle on compact quartets with O(1e-2) integrals."""
    from paper_2605_10312_gb300.gen import verify
    prog = program.make(4, 4, 4, 4)
    deep, _ = coop.choose_both(prog)
    assert (deep.T, deep.ilp, deep.lag) == coop.WIDEST_SHAPE + (1,) and int(deep.steps1.max()) == 4
    # Phase 2 in waves of up to eight steps
    assert int(deep.steps2.max()) == 8
    assert verify.verify_coop(deep, prog.L, len(encode.coef_table())) == []
    basis, q = synth.class_sweep((4, 4, 4, 4), 2, kset=(1, 2), seed=24, box_angstrom=0.5, exp_range=(0.3, 3.0))
    ref, _ = blocks(basis, q)
    ref = ref.reshape(q.shape[0], -1)
    assert np.abs(ref).max() > 1e-2
    got = run_coop(deep, prog, basis, q)
    assert within(got, ref).all()


def test_split_barrier_schedule_keeps_adjacent_waves_apart():
    """With split barriers a node's parents lie at least two waves back and a
    slot is reused two waves after its last read, so nothing one wave writes
    is read or written by the next (a lane may run wave w + 1 while another
    still runs wave w)."""
    g = vrr.build(2, 2, 2, 1)
    order = vrr.schedule(g)
    pos = np.empty(len(g), dtype=np.int64)
    pos[np.array(order)] = np.arange(len(g))
    par = [[p for _, p in ts] for ts in g.terms]
    waves = coop.wave_schedule(par, pos, 32, lag=2)
    wave_of = {v: w for w, vs in enumerate(waves) for v in vs}
    assert len(wave_of) == len(g)
    for v, ps in enumerate(par):
        for p in ps:
            assert wave_of[p] <= wave_of[v] - 2
    slot, n = coop.allocate_over_waves(par, waves, np.ones(len(g), dtype=bool), lag=2)
    last = {v: max([wave_of[c] for c, ps in enumerate(par) if v in ps], default=wave_of[v]) for v in range(len(g))}
    owners = {}
    for v in sorted(range(len(g)), key=lambda v: wave_of[v]):
        s = int(slot[v])
        if s in owners:
            assert last[owners[s]] + 2 <= wave_of[v]
        owners[s] = v


@pytest.mark.parametrize("T,ilp", [(64, 2), (128, 2), (128, 4), (256, 2)])
@pytest.mark.parametrize("ls", [(1, 1, 1, 1), (2, 2, 1, 1), (3, 1, 2, 0), (2, 2, 2, 1)])
def test_split_barrier_programs_match_oracle(ls, T, ilp):
    """Split-barrier programs reproduce the oracle wave by wave, and the
    verifier finds no hazard between adjacent waves."""
    from paper_2605_10312_gb300.gen import verify
    prog = program.make(*ls)
    cp = coop.build(prog, T, ilp, 1, lag=2)
    assert cp.lag == 2
    assert verify.verify_coop(cp, prog.L, len(encode.coef_table())) == []
    basis, q = synth.class_sweep(ls, 3, kset=(1, 2), seed=29, box_angstrom=3.0, exp_range=(0.1, 30))
    ref, _ = blocks(basis, q)
    got = run_coop(cp, prog, basis, q)
    assert within(got, ref.reshape(q.shape[0], -1)).all()


def test_verifier_catches_adjacent_wave_hazards():
    """A full-barrier program read as a split-barrier one has values that the
    next wave reads; the verifier reports that, and a planted in-wave
    read-after-write conflict too."""
    import copy
    from paper_2605_10312_gb300.gen import verify
    prog = program.make(2, 2, 1, 1)
    ncoef = len(encode.coef_table())
    cp = coop.build(prog, 64, 2)
    assert verify.verify_coop(cp, prog.L, ncoef) == []
    c = copy.deepcopy(cp)
    c.lag = 2
    assert any("split barriers" in m for m in verify.verify_coop(c, prog.L, ncoef))
    # in one wave: make a node write the slot another node of the wave reads
    c = copy.deepcopy(cp)
    W = c.T * c.ilp
    w0 = c.ph1[:int(c.steps1[0]) * W]
    for wv in range(1, len(c.steps1)):
        lo = int(np.sum(c.steps1[:wv])) * W
        blk = c.ph1[lo:lo + int(c.steps1[wv]) * W]
        meta = blk[:, 3] >> 16
        term = np.flatnonzero((meta & 0xC000) == 0)
        keep = np.flatnonzero(((meta & 0x8000) == 0) & ((blk[:, 0] & 0xFFFF) != 0xFFFF))
        if term.size and keep.size:
            src = int(blk[term[0], 1] & 0xFFFF)
            i = lo + int(keep[0])
            c.ph1[i, 0] = (c.ph1[i, 0] & 0xFFFF0000) | src
            break
    assert any("reads a slot it writes" in m for m in verify.verify_coop(c, prog.L, ncoef))


def test_half_warp_wavefront_model():
    """64-bit shared accesses: a half-warp of 16 lanes reading 16 words in
    16 distinct bank pairs takes one wavefront; 16 words in one bank pair
    take 16; one repeated word is a broadcast; masked lanes take none."""
    ids = np.arange(32).reshape(1, 32)
    on = np.ones_like(ids, dtype=bool)
    assert coop._half_warp_wavefronts(ids, on) == (2, 2)
    assert coop._half_warp_wavefronts(ids * 16, on) == (32, 2)
    assert coop._half_warp_wavefronts(np.zeros_like(ids), on) == (2, 2)
    half = on.copy()
    half[0, 16:] = False
    assert coop._half_warp_wavefronts(ids * 16, half) == (16, 1)
    assert coop._half_warp_wavefronts(ids, np.zeros_like(on)) == (0, 0)


@pytest.mark.parametrize("ls,T,ilp,k1,k2", [((2, 2, 2, 2), 64, 2, 1, 2), ((3, 3, 2, 2), 128, 2, 1, 4),
                                          ((3, 2, 2, 1), 32, 2, 1, 4)])
def test_bank_aware_slots(ls, T, ilp, k1, k2):
    """Bank-aware slot choice keeps the slot count, lowers the modelled
    shared-memory wavefronts of both phases, passes the bounds and hazard
    verifier, and the program still reproduces the oracle."""
    from paper_2605_10312_gb300.gen import verify
    prog = program.make(*ls)
    plain = coop.build(prog, T, ilp, k1, wave_steps2=k2)
    banked = coop.build(prog, T, ilp, k1, wave_steps2=k2, banked=True, h_shared=True)
    assert banked.nslot == plain.nslot
    a, b = coop.shared_wavefronts(plain, True), coop.shared_wavefronts(banked, True)
    assert b[1] == a[1] and b[3] == a[3]          # same instructions
    assert b[0] < a[0] and b[2] < a[2]
    assert verify.verify_coop(banked, prog.L, len(encode.coef_table())) == []
    basis, q = synth.class_sweep(ls, 3, kset=(1, 2), seed=29, box_angstrom=3.0, exp_range=(0.1, 30))
    ref, _ = blocks(basis, q)
    got = run_coop(banked, prog, basis, q)
    assert within(got, ref.reshape(q.shape[0], -1)).all()


def test_largest_global_tier_program_fits_the_fixed_scratch():
    """eri_compute_fixed_scratch refuses a class whose global-scratch
    program needs more than its 64 MiB array for one 128-thread block
    (slots x 128 threads x 8 bytes).  The largest class, (gg|gg), needs about
    41 MB, so every class of the library (l <= 4) is accepted and the
    refusal is reachable only by larger programs."""
    enc = encode.encode(program.make(4, 4, 4, 4))
    need = enc.nslot * 128 * 8
    assert 32 << 20 < need <= 64 << 20, need
