"""The arithmetic that makes the sliced tensor-core compose exact, checked on the CPU with an
independent numpy restatement of error-free splitting (Ozaki, Ogita, Oishi & Rump, 2012):
values scaled by a power of two to |x| <= 1 are written as 8 balanced base-64 digits.

Pinned here, against the arithmetic itself rather than the CUDA code:
  * the digits are integers with |d_1| <= 64 and |d_s| <= 32, which BF16 holds exactly;
  * the residual after 8 digits is at most 2^-49;
  * for the diagonal s + t of the digit-plane products, the per-term bound sum |a_s||b_t|
    times the fan-in K stays at or below 2^24 (the FP32 accumulator adds integers exactly) up
    to K = 1638, the library's limit, and not beyond;
  * the products summed per diagonal and combined with their scales reproduce the FP64 dot
    product to within (3 K + 1) 2^-48 of the scales.
"""
import numpy as np

BETA, PLANES = 6, 8


def digits(x):
    """Balanced base-2^BETA digits of x (|x| <= 1), nearest-digit recursion, and the residual."""
    d = []
    r = np.array(x, dtype=np.float64)
    for _ in range(PLANES):
        t = np.ldexp(r, BETA)
        q = np.rint(t)
        d.append(q)
        r = t - q
    return np.array(d), np.ldexp(r, -BETA * PLANES)


def scaled(v, axis):
    m = np.max(np.abs(v), axis=axis, keepdims=True)
    e = np.where(m > 0, np.ceil(np.log2(np.where(m > 0, m, 1.0))), 0.0)
    return np.ldexp(v, -e.astype(int)), e


def test_digit_bounds_and_residual():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-1, 1, 200000), [1.0, -1.0, 0.5, -0.5, 1 - 2**-53, 2**-60, 0.0]])
    d, res = digits(x)
    assert np.all(d == np.rint(d))
    assert np.abs(d[0]).max() <= 64 and np.abs(d[1:]).max() <= 32
    # reconstruction: x = sum d_s 2^-6s + residual, exactly
    rec = sum(np.ldexp(d[s], -BETA * (s + 1)) for s in range(PLANES))
    assert np.array_equal(rec + res, x)
    assert np.abs(res).max() <= 2.0**-49
    # BF16 holds every digit exactly: 8 significant bits cover |d| <= 256
    import torch
    t = torch.tensor(d.ravel(), dtype=torch.float64)
    assert torch.equal(t.to(torch.bfloat16).to(torch.float64), t)


def _diagonal_term_bound(dg):
    """max over digit pairs (s, t), s + t = dg (0-based planes), of sum |a_s| |b_t|."""
    bound = lambda s: 64 if s == 0 else 32
    return sum(bound(s) * bound(dg - s) for s in range(PLANES) if 0 <= dg - s < PLANES)


def test_diagonal_sums_fit_fp32_up_to_the_fan_in_limit():
    worst = max(_diagonal_term_bound(dg) for dg in range(PLANES))
    assert worst == 10240
    assert 1638 * worst <= 2**24 < 1639 * worst


def test_sliced_dot_products_match_fp64_within_the_bound():
    rng = np.random.default_rng(1)
    for K in (3, 64, 512, 1638):
        W = rng.normal(0, 1 / np.sqrt(K), (16, K))
        Z = rng.normal(0, 1, (K, 8)) * (rng.random((K, 8)) < 0.5)      # masked columns
        Ws, eA = scaled(W, 1)
        Zs, eB = scaled(Z, 0)
        a, _ = digits(Ws)
        b, _ = digits(Zs)
        # each diagonal's sum of digit-plane products, as the FP32 accumulator holds it
        acc = np.zeros((PLANES, 16, 8))
        for s in range(PLANES):
            for t in range(PLANES - s):
                acc[s + t] += a[s] @ b[t]
        assert np.all(np.abs(acc) <= 2**24)
        assert np.array_equal(acc.astype(np.float32).astype(np.float64), acc)     # FP32-exact integers
        val = sum(np.ldexp(acc[dg], -BETA * (dg + 2)) for dg in range(PLANES))
        got = np.ldexp(val, (eA + eB).astype(int))
        ref = W @ Z
        bound = (3 * K + 1) * 2.0**-48 * np.ldexp(1.0, (eA + eB).astype(int))
        assert np.all(np.abs(got - ref) <= bound + 4 * np.finfo(float).eps * np.abs(W) @ np.abs(Z))
