"""The FP32 primitive-quartet set-up of mixed-precision plans, emulated on
the CPU with numpy float32 arithmetic (the operations of the device's FP32
set-up in its order; the device fuses two multiply-adds of T, one rounding
fewer each): P - Q from the two-float form of P
keeps FP32 relative accuracy for close pairs far from the origin, where a
plain float P loses it to cancellation; W - P, W - Q, T and the prefactor
then stay within a few FP32 roundings of their FP64 values."""
import numpy as np

F = np.float32
EPS = 2.0 ** -24


def split(p):
    """The pair set-up's FP32 form of P: P_hi + P_lo."""
    hi = p.astype(F)
    lo = (p - hi.astype(np.float64)).astype(F)
    return hi, lo


def pq_two_float(p, q):
    ph, pl = split(p)
    qh, ql = split(q)
    return (ph - qh) + (pl - ql)          # float32 throughout


def setup_f32(zb, zk, p, q, kb, kk):
    """s, W - P, W - Q, T and the prefactor as the FP32 set-up forms them."""
    zb, zk, kb, kk = F(zb), F(zk), F(kb), F(kk)
    s = F(1.0) / (zb + zk)
    te, tz = zk * s, zb * s
    pq = pq_two_float(p, q)
    wp, wq = -te * pq, tz * pq
    rho = zb * te
    t = rho * (pq[0] * pq[0] + pq[1] * pq[1] + pq[2] * pq[2])
    pref = kb * kk * np.sqrt(s, dtype=F)
    return s, wp, wq, t, pref


def test_two_float_p_keeps_relative_accuracy_of_close_pairs():
    rng = np.random.default_rng(3)
    worst_split = worst_plain = 0.0
    for _ in range(2000):
        p = rng.uniform(-30.0, 30.0, 3)                     # bohr, a large cluster
        q = p + rng.uniform(-1.0, 1.0, 3) * 10.0 ** rng.uniform(-5, 0)
        exact = p - q
        a = pq_two_float(p, q).astype(np.float64)
        b = (p.astype(F) - q.astype(F)).astype(np.float64)
        # two floats hold P to about 48 bits: an absolute floor of |P| 2^-47
        # beside one rounding of the difference itself
        floor = np.max(np.abs(p)) * 2.0 ** -47
        rel = lambda x: np.max(np.abs(x - exact) / (np.abs(exact) + floor / EPS))
        worst_split = max(worst_split, rel(a))
        worst_plain = max(worst_plain, rel(b))
    assert worst_split <= 3 * EPS
    assert worst_plain > 1e-3          # the cancellation the two-float form avoids


def test_fp32_setup_within_a_few_roundings_of_fp64():
    rng = np.random.default_rng(4)
    for _ in range(500):
        zb, zk = 10.0 ** rng.uniform(-1, 3, 2)
        kb, kk = 10.0 ** rng.uniform(-3, 2, 2)
        p = rng.uniform(-30.0, 30.0, 3)
        q = p + rng.uniform(-3.0, 3.0, 3)
        s, wp, wq, t, pref = setup_f32(zb, zk, p, q, kb, kk)
        s64 = 1.0 / (zb + zk)
        pq = p - q
        wp64, wq64 = -zk * s64 * pq, zb * s64 * pq
        t64 = zb * zk * s64 * np.dot(pq, pq)
        pref64 = kb * kk * np.sqrt(s64)
        # EPS is the unit roundoff: rounding the inputs to float and every
        # FP32 operation each add at most one EPS of relative error
        assert abs(s - s64) <= 4 * EPS * s64
        assert np.all(np.abs(wp - wp64) <= 16 * EPS * np.abs(wp64))
        assert np.all(np.abs(wq - wq64) <= 16 * EPS * np.abs(wq64))
        assert abs(t - t64) <= 32 * EPS * t64
        assert abs(pref - pref64) <= 12 * EPS * pref64
