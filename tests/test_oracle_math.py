"""Pins of the oracle's elementary functions and random numbers.

The particle path must be bit-reproducible, so the oracle carries its own
exp, log, logf, sin/cos(2 pi u) and Philox4x64-10.  These are pinned to
independent implementations: numpy's Philox bit generator (an independent
implementation of the same published generator) and the platform libm /
mpmath, within 2 ulp.
"""
import numpy as np
import pytest

import oracle


def _ulp_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(got - ref) / np.spacing(np.abs(ref))


@pytest.mark.parametrize("key", [(0, 0), (1, 0), (5, 7), (2**64 - 1, 12345)])
def test_philox_matches_numpy(key):
    rng = np.random.default_rng(11)
    for _ in range(50):
        ctr = rng.integers(1, 2**63, size=4, dtype=np.uint64)
        # numpy increments the 256-bit counter before each block
        prev = ctr.copy()
        prev[0] -= np.uint64(1)
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=prev)
        ref = bg.random_raw(4)
        got = oracle.philox(ctr, key)
        assert np.array_equal(got, ref)


def test_philox_counter_words_all_matter():
    base = oracle.philox([3, 4, 5, 6], [9, 0])
    for w in range(4):
        c = [3, 4, 5, 6]
        c[w] += 1
        assert not np.array_equal(oracle.philox(c, [9, 0]), base)


def test_exp_within_2ulp():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-745.0, 709.7, 400000), rng.uniform(-1, 1, 200000),
                        rng.uniform(-1e-8, 1e-8, 20000), [0.0, 1.0, -1.0, 709.7, -708.0, -740.0]])
    y = oracle.math_d("exp", x)
    ref = np.exp(x)
    normal = ref > 2.3e-308
    assert _ulp_err(y[normal], ref[normal]).max() <= 2.0
    # gradual underflow region: absolute error within 2 units of the smallest subnormal grid
    sub = ~normal & (ref > 0)
    assert np.all(np.abs(y[sub] - ref[sub]) <= 2 * 5e-324)
    assert oracle.math_d("exp", np.array([-800.0, 800.0, 0.0]))[0] == 0.0
    assert np.isinf(oracle.math_d("exp", np.array([800.0]))[0])
    assert oracle.math_d("exp", np.array([0.0]))[0] == 1.0


def test_log_within_2ulp():
    rng = np.random.default_rng(2)
    x = np.concatenate([10.0 ** rng.uniform(-300, 300, 300000), rng.uniform(0.5, 2.0, 200000),
                        rng.uniform(1 - 1e-6, 1 + 1e-6, 50000), np.array([5e-324, 1e-310, 2.2e-308]),
                        rng.uniform(1e-300, 1.0, 100000)])
    y = oracle.math_d("log", x)
    ref = np.log(x)
    nz = ref != 0
    assert _ulp_err(y[nz], ref[nz]).max() <= 2.0
    assert oracle.math_d("log", np.array([1.0]))[0] == 0.0
    # uniforms of the particle path: eta = (k + 1/2) 2^-53
    k = rng.integers(0, 2**53, 100000, dtype=np.int64).astype(np.float64)
    eta = (k + 0.5) * 2.0 ** -53
    assert _ulp_err(oracle.math_d("log", eta), np.log(eta)).max() <= 2.0


def test_logf_within_2ulp():
    rng = np.random.default_rng(3)
    x = np.concatenate([(10.0 ** rng.uniform(-37, 37, 200000)), rng.uniform(0.5, 2.0, 200000),
                        ((np.arange(1, 2**23, 97) + 0.5) * 2.0 ** -23)]).astype(np.float32)
    y = oracle.logf(x).astype(np.float64)
    ref64 = np.log(x.astype(np.float64))
    ref = ref64.astype(np.float32).astype(np.float64)
    nz = ref != 0
    ulp32 = np.spacing(np.abs(ref[nz]).astype(np.float32)).astype(np.float64)
    assert (np.abs(y[nz] - ref64[nz]) / ulp32).max() <= 2.0


def test_sincos2pi_within_2ulp():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(4)
    k = rng.integers(0, 2**53, 4000, dtype=np.int64).astype(np.float64)
    u = np.concatenate([(k + 0.5) * 2.0 ** -53, [0.0, 0.125, 0.25, 0.375, 0.5, 0.75, 0.999999]])
    s = oracle.math_d("sin2pi", u)
    c = oracle.math_d("cos2pi", u)
    rs = np.array([float(mpmath.sin(2 * mpmath.pi * mpmath.mpf(v))) for v in u])
    rc = np.array([float(mpmath.cos(2 * mpmath.pi * mpmath.mpf(v))) for v in u])
    for got, ref in ((s, rs), (c, rc)):
        big = np.abs(ref) > 1e-300
        err = np.abs(got[big] - ref[big]) / np.spacing(np.abs(ref[big]))
        # near a zero of the function the absolute error is set by the argument
        err_abs = np.abs(got[big] - ref[big]) <= 4e-16
        assert np.all((err <= 2.0) | err_abs)
    assert np.allclose(s * s + c * c, 1.0, rtol=0, atol=4e-16)


def test_sincos2pi_f_against_libm_and_symmetry():
    """Binary32 sin/cos(2 pi u) of the mixed-mode particles: within 3 binary32
    ulps of the double-precision libm value (absolute 6e-8 near a zero), the
    exact quarter-turn values, and the exact symmetry u -> 1 - u that a wrong
    quadrant rotation or sign would break."""
    k = np.arange(0, 2**23, 37, dtype=np.int64)
    u = ((k + 0.5) * 2.0 ** -23).astype(np.float32)
    s, c = oracle.sincos2pi_f(u)
    ang = 2.0 * np.pi * u.astype(np.float64)
    for got, ref in ((s, np.sin(ang)), (c, np.cos(ang))):
        ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
        err = np.abs(got.astype(np.float64) - ref)
        assert np.all((err <= 3.0 * ulp) | (err <= 6e-8))
    assert np.abs(s.astype(np.float64) ** 2 + c.astype(np.float64) ** 2 - 1.0).max() < 3e-7
    q = np.array([0.0, 0.25, 0.5, 0.75], dtype=np.float32)
    sq, cq = oracle.sincos2pi_f(q)
    assert np.array_equal(np.abs(sq), [0.0, 1.0, 0.0, 1.0]) and np.array_equal(np.abs(cq), [1.0, 0.0, 1.0, 0.0])
    assert sq[1] == 1.0 and sq[3] == -1.0 and cq[0] == 1.0 and cq[2] == -1.0
    s2, c2 = oracle.sincos2pi_f((1.0 - u.astype(np.float64)).astype(np.float32))
    assert np.array_equal(s2, -s) and np.array_equal(c2, c)


def test_philox32_mixes_every_input_word():
    """Philox4x32-10 (the free-transport-time draw): every counter and key word
    changes about half of the 128 output bits; outputs of consecutive counters
    are uniform words.  The exact bits are pinned against an independent
    implementation (cuRAND's) in the GPU suite."""
    base_c, base_k = np.array([5, 7, 11, 1], dtype=np.uint32), np.array([3, 9], dtype=np.uint32)
    ref = oracle.philox32(base_c, base_k)
    flips = []
    for which in range(6):
        for bit in (0, 13, 31):
            c, k = base_c.copy(), base_k.copy()
            if which < 4:
                c[which] ^= np.uint32(1 << bit)
            else:
                k[which - 4] ^= np.uint32(1 << bit)
            out = oracle.philox32(c, k)
            flips.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(out, ref)))
    assert 40 < np.mean(flips) < 88 and min(flips) > 20
    words = np.array([oracle.philox32([i, 0, 0, 1], [1, 0]) for i in range(4096)], dtype=np.float64)
    u = (words.ravel() + 0.5) / 2.0 ** 32
    from scipy import stats
    assert stats.kstest(u, "uniform").pvalue > 1e-4
