"""GPU parity of ffgpu_fgemm against the CPU oracle, bit for bit.

Sizes are chosen so that the oracle finishes in seconds while the kernel still
crosses several tiles (128 x 256), several 512-long chunks of the inner
dimension (in-place reductions), ragged tails in every dimension, more tiles
than SMs (several tiles per persistent CTA) and both parities of the channel
count (jobs paired across tiles).  The full-size configuration is checked on
sampled entries and by Freivalds' test.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_cs_0601133_gb300 as ff
from paper_cs_0601133_gb300 import workloads as W
from tests.gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu

@pytest.fixture(autouse=True, scope="module")
def tensor_cores_only():
    """Every product of this module on the tensor-core route, small ones
    included (ffgpu_fgemm would send those to the CUDA-core kernel)."""
    old = ff.get_small_threshold()
    ff.set_small_threshold(0)
    yield
    ff.set_small_threshold(old)


SWEEP = [251, 65521, 8388593, 2147483647]


def run(A, B, C, p, alpha, beta, pad=0):
    dA, dB, dC = to_dev(A, pad), to_dev(B, pad), to_dev(C, pad)
    ff.fgemm(dA, dB, p, alpha, beta, dC)
    torch.cuda.synchronize()
    assert ff.last_device_error() == 0
    return from_dev(dC)


def check(A, B, C, p, alpha, beta, pad=0):
    got = run(A, B, C, p, alpha, beta, pad)
    expect = oracle.fgemm(A, B, p, alpha, beta, C)
    if not np.array_equal(got, expect):
        bad = np.argwhere(got != expect)
        i, j = bad[0]
        raise AssertionError("p=%d shape=%s: %d mismatches, first at (%d,%d): got %d expect %d"
                             % (p, (A.shape, B.shape), len(bad), i, j, got[i, j], expect[i, j]))


def test_config1_512_cube_p65521():
    A, B, C, _, _ = W.square_problem(512, 65521, with_alpha_beta=False)
    check(A, B, C, 65521, 1, 0)


@pytest.mark.parametrize("p", SWEEP + [2, 3, 256, 257, 1000003])
def test_random_words_alpha_beta(p):
    rng = W.rng_for("square", 11, p)
    m, k, n = 300, 1100, 520          # ragged in every dimension, 3 chunks of k
    A = W.uniform_words(rng, (m, k))
    B = W.uniform_words(rng, (k, n))
    C = W.uniform_words(rng, (m, n))
    alpha, beta = int(rng.integers(0, 2**32)), int(rng.integers(0, 2**32))
    check(A, B, C, p, alpha, beta)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 7, 3), (129, 65, 257), (127, 64, 255),
                                   (128, 512, 256), (256, 513, 512), (5, 2000, 9)])
@pytest.mark.parametrize("p", [65521, 2147483647])
def test_ragged_shapes(shape, p):
    m, k, n = shape
    rng = W.rng_for("square", 12, m * 7 + k * 3 + n)
    A = W.uniform_residues(rng, (m, k), p)
    B = W.uniform_residues(rng, (k, n), p)
    C = W.uniform_residues(rng, (m, n), p)
    check(A, B, C, p, 3, 5)


@pytest.mark.parametrize("p", SWEEP)
def test_padded_leading_dimensions(p):
    rng = W.rng_for("square", 13, p)
    A = W.uniform_residues(rng, (200, 300), p)
    B = W.uniform_residues(rng, (300, 270), p)
    C = W.uniform_residues(rng, (200, 270), p)
    check(A, B, C, p, 7, 11, pad=5)


@pytest.mark.parametrize("p", SWEEP)
@pytest.mark.parametrize("k", [512, 2048, 4096])
def test_adversarial_all_p_minus_1(p, k):
    m, n = 256, 512
    A, B, C = W.adversarial_problem(m, n, k, p)
    alpha, beta = p - 1, p - 1
    got = run(A, B, C, p, alpha, beta)
    # closed form: (p-1)^2 = 1 mod p, so A*B = k*J and the result is alpha*k + beta*(p-1)
    expect = (alpha * k + beta * (p - 1)) % p
    assert np.all(got == expect)


@pytest.mark.parametrize("p", [2147483647, 65521])
def test_many_tiles_per_cta(p):
    # 16 x 16 tiles > SM count: every persistent CTA walks several tiles
    m, n, k = 2048, 4096, 256
    rng = W.rng_for("square", 14, p)
    A = W.uniform_residues(rng, (m, k), p)
    B = W.uniform_residues(rng, (k, n), p)
    C = W.uniform_residues(rng, (m, n), p)
    check(A, B, C, p, 2, 3)


def test_odd_and_even_channel_counts():
    # p < 2^31 with k = 512 needs 9 channels (odd: jobs pair across tiles), k = 1024 needs 10
    p = 2147483647
    assert ff.fgemm_plan(1, 1, 512, p)["channels"] % 2 == 1
    for k in (512, 1024):
        rng = W.rng_for("square", 15, k)
        A = W.uniform_residues(rng, (600, k), p)
        B = W.uniform_residues(rng, (k, 1100), p)
        C = W.uniform_residues(rng, (600, 1100), p)
        check(A, B, C, p, 1, 1)


def test_k_zero_and_empty():
    p = 65521
    rng = W.rng_for("square", 16)
    C = W.uniform_words(rng, (33, 47))
    got = run(np.zeros((33, 0), np.uint32), np.zeros((0, 47), np.uint32), C, p, 9, 10)
    assert np.array_equal(got, (10 * C.astype(np.uint64) % p).astype(np.uint32))
    dC = to_dev(C)
    assert ff.fgemm_ptr(0, 47, 5, p, 1, 0, 5, 0, 47, 0, dC.data_ptr(), 47) == 0


def test_caller_workspace_matches_pool():
    p = 8388593
    rng = W.rng_for("square", 17)
    A = W.uniform_residues(rng, (300, 700), p)
    B = W.uniform_residues(rng, (700, 400), p)
    C = W.uniform_residues(rng, (300, 400), p)
    ws_bytes = ff.fgemm_workspace_size(300, 400, 700, p)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    dA, dB, dC = to_dev(A), to_dev(B), to_dev(C)
    ff.fgemm_ws(dA, dB, p, 5, 6, dC, ws)
    torch.cuda.synchronize()
    assert np.array_equal(from_dev(dC), oracle.fgemm(A, B, p, 5, 6, C))
    small = torch.empty(ws_bytes // 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(ff.FFGPUError):
        ff.fgemm_ws(dA, dB, p, 5, 6, dC, small)


@pytest.mark.parametrize("p", [65521, 2147483647])
def test_full_size_8192_sampled(p):
    """The bench configuration (n = 8192, alpha, beta uniform): 4096 sampled
    entries recomputed by the oracle, plus Freivalds' test on the whole C."""
    n = 8192
    A, B, C, alpha, beta = W.square_problem(n, p)
    got = run(A, B, C, p, alpha, beta)
    rng = np.random.default_rng(5)
    rows = rng.integers(0, n, 4096)
    cols = rng.integers(0, n, 4096)
    # include the corners and the last tile's ragged edges
    rows[:4] = [0, 0, n - 1, n - 1]
    cols[:4] = [0, n - 1, 0, n - 1]
    expect = oracle.fgemm_entries(A, B, p, alpha, beta, C, rows, cols)
    assert np.array_equal(got[rows, cols], expect)
    assert oracle.freivalds(A, B, C, got, p, alpha, beta, trials=2)


@pytest.mark.parametrize("p", [251, 2147483647])
def test_full_size_16384_sampled(p):
    """The sweep's largest order (n = 16384, 1 GiB per matrix): sampled
    entries recomputed by the oracle (random ones, and runs along the last
    row and the last column), and Freivalds' test on the whole C."""
    n = 16384
    A, B, C, alpha, beta = W.square_problem(n, p)
    got = run(A, B, C, p, alpha, beta)
    rng = np.random.default_rng(16384)
    edge = np.arange(n - 512, n)
    rows = np.concatenate([rng.integers(0, n, 2048), np.full(512, n - 1), edge])
    cols = np.concatenate([rng.integers(0, n, 2048), edge, np.full(512, n - 1)])
    expect = oracle.fgemm_entries(A, B, p, alpha, beta, C, rows, cols)
    assert np.array_equal(got[rows, cols], expect)
    assert oracle.freivalds(A, B, C, got, p, alpha, beta, trials=2)


@pytest.mark.parametrize("kernel", ["single", "pair"])
@pytest.mark.parametrize("shape,p", [((300, 1100, 520), 2147483647), ((129, 65, 257), 65521),
                                     ((2048, 256, 4096), 2147483647), ((600, 512, 1100), 2147483647),
                                     ((256, 2048, 512), 251)])
def test_both_tensor_core_kernels(kernel, shape, p, monkeypatch):
    """The one-CTA kernel (128 x 256 tiles) and the CTA-pair kernel (256 x 256
    tiles, cta_group::2) must both be exact on ragged shapes, several tiles
    per CTA, odd channel counts and long inner dimensions."""
    monkeypatch.setenv("FFGPU_KERNEL", kernel)
    m, k, n = shape
    rng = W.rng_for("square", 20, m + k + n, p)
    A = W.uniform_words(rng, (m, k))
    B = W.uniform_words(rng, (k, n))
    C = W.uniform_words(rng, (m, n))
    check(A, B, C, p, 5, 7)


@pytest.mark.parametrize("kernel", ["single", "pair"])
def test_both_kernels_adversarial(kernel, monkeypatch):
    monkeypatch.setenv("FFGPU_KERNEL", kernel)
    p = 2147483647
    m, n, k = 512, 512, 4096
    A, B, C = W.adversarial_problem(m, n, k, p)
    got = run(A, B, C, p, p - 1, p - 1)
    assert np.all(got == ((p - 1) * k + (p - 1) * (p - 1)) % p)


# ---------------------------------------------------------------------------
# Worst cases of the two bounds the product rests on (section 2.1.2, eqs. 1-2,
# restated for this design): (1) every partial sum of a channel's f32
# accumulator is an integer below 2^24 between two in-place reductions, and
# (2) the integer value |X| of a product entry stays within M/4, M the product
# of the plan's moduli, where the reconstruction from the residues is exact.
# Inputs of all-(p-1) do not reach either bound (p - 1 is centred to -1, so
# every product is 1); the inputs below do, with the sign pattern of
# workloads.sign_pattern_problem so that every sum grows monotonically.
# ---------------------------------------------------------------------------

def balanced(x: int, m: int) -> int:
    r = x % m
    return r - m if r > m // 2 else r


def closed_form(s, t, k, a, b, p, alpha, beta, C):
    """(alpha s_i t_j k a b + beta C) mod p, entry by entry, in Python integers."""
    v = [(alpha * k * a * b) % p, (-alpha * k * a * b) % p]
    X = np.where(np.outer(s, t) > 0, v[0], v[1]).astype(np.uint64)
    return ((X + (beta % p) * C.astype(np.uint64)) % p).astype(np.uint32)


def check_sampled(A, B, C, got, p, alpha, beta, seed, count=512):
    rng = np.random.default_rng(seed)
    m, n = got.shape
    rows = np.concatenate([rng.integers(0, m, count), [0, m - 1, m - 1]])
    cols = np.concatenate([rng.integers(0, n, count), [n - 1, 0, n - 1]])
    expect = oracle.fgemm_entries(A, B, p, alpha, beta, C, rows, cols)
    assert np.array_equal(got[rows, cols], expect)


def largest_x_with_half_residues(p, moduli):
    """x = -1/2 modulo the product of the leading moduli, as many of them as
    keep x <= floor(p/2) (so that x is its own centred representative): the
    balanced residue of x is +(m_c - 1)/2 in each of those channels."""
    Mx, used = 1, 0
    for mc in moduli:
        if (Mx * mc - 1) // 2 > p // 2:
            break
        Mx *= mc
        used += 1
    assert used >= 1
    return (Mx - 1) // 2, used


@pytest.mark.parametrize("kernel", ["single", "pair"])
@pytest.mark.parametrize("p", [65521, 8388593, 2147483647])
def test_chunk_sums_reach_the_accumulator_bound(kernel, p, monkeypatch):
    """Residues at +-(m_c - 1)/2 in the largest moduli (255, 253, ...): with
    the sign pattern each chunk of a channel's accumulator sums chunk * 127^2
    (channel 255) before the in-place reduction, 98 % of 2^24."""
    monkeypatch.setenv("FFGPU_KERNEL", kernel)
    m, n = 300, 520
    plan = ff.fgemm_plan(m, n, 4096, p)
    chunk, mods = plan["k_chunk"], plan["moduli"]
    k = 3 * chunk + 300                        # three full chunks and a ragged one
    plan = ff.fgemm_plan(m, n, k, p)
    assert plan["k_chunk"] == chunk and plan["mode"] == 2
    x, used = largest_x_with_half_residues(p, plan["moduli"])
    assert all(balanced(x, mc) == (mc - 1) // 2 for mc in plan["moduli"][:used])
    # host side: the chunk sum this input implies in each channel, plus the
    # carried reduced value (at most (m_c + 1)/2)
    peak = max(chunk * balanced(x, mc) ** 2 + (mc + 1) // 2 for mc in plan["moduli"])
    assert 0.98 * 2**24 <= peak < 2**24, peak
    rng = W.rng_for("worstcase", 1, p)
    A, B, C, s, t = W.sign_pattern_problem(rng, m, n, k, p, x, x)
    alpha, beta = int(rng.integers(1, p)), int(rng.integers(0, p))
    got = run(A, B, C, p, alpha, beta)
    assert np.array_equal(got, oracle.fgemm(A, B, p, alpha, beta, C))
    assert np.array_equal(got, closed_form(s, t, k, x, x, p, alpha, beta, C))


@pytest.mark.parametrize("kernel", ["single", "pair"])
@pytest.mark.parametrize("p,v", [(251, 125), (255, 127), (253, 126), (3, 1)])
def test_direct_mode_chunk_sums_at_the_bound(kernel, p, v, monkeypatch):
    """One channel, the modulus p itself (p <= 255): entries +-floor(p/2), the
    largest centred magnitude, so each chunk sums chunk * floor(p/2)^2 (for
    p = 255: 1024 * 127^2 = 98.4 % of 2^24); three chunks and a ragged one."""
    monkeypatch.setenv("FFGPU_KERNEL", kernel)
    m, n = 260, 300
    plan = ff.fgemm_plan(m, n, 4096, p)
    assert plan["mode"] == 1 and plan["channels"] == 1
    chunk = plan["k_chunk"]
    k = 3 * chunk + 100
    peak = chunk * v * v + v + 1
    assert peak < 2**24
    if p >= 251:
        assert peak >= 0.95 * 2**24, peak
    rng = W.rng_for("worstcase", 2, p)
    A, B, C, s, t = W.sign_pattern_problem(rng, m, n, k, p, v, v)
    got = run(A, B, C, p, p - 1, 7)
    assert np.array_equal(got, oracle.fgemm(A, B, p, p - 1, 7, C))
    assert np.array_equal(got, closed_form(s, t, k, v, v, p, p - 1, 7, C))


def channel_boundaries(p, k_hi):
    """(c, k_max) for every channel count c the plan uses below k_hi: k_max is
    the longest inner dimension summed with c channels (found by bisection on
    the plan, a host-side call)."""
    out = []
    k = 1
    while k <= k_hi:
        c = ff.fgemm_plan(1, 1, k, p)["channels"]
        lo, hi = k, k_hi + 1
        while hi - lo > 1:                      # largest k with the same count
            mid = (lo + hi) // 2
            if ff.fgemm_plan(1, 1, mid, p)["channels"] == c:
                lo = mid
            else:
                hi = mid
        if lo < k_hi:
            out.append((c, lo))
        k = lo + 1
    return out


BOUNDARY_CASES = [(p, which) for p in (65521, 8388593, 2147483647) for which in (-2, -1)]


@pytest.mark.parametrize("kernel", ["single", "pair"])
@pytest.mark.parametrize("p,which", BOUNDARY_CASES)
@pytest.mark.parametrize("past", [0, 1])
def test_reconstruction_at_the_channel_boundaries(kernel, p, which, past, monkeypatch):
    """Entries +-floor(p/2) (the largest centred magnitude) with the sign
    pattern, so every entry of the product is +-k floor(p/2)^2.  At the
    longest k a channel count admits (past = 0) that is at least 3/4 of M/4,
    the reconstruction's limit; one more (past = 1) switches to the next
    channel count.  The two largest switches below 200000 per prime (for
    2^31 - 1: 9 -> 10 channels at k = 605 and 10 -> 11 at k = 134930)."""
    monkeypatch.setenv("FFGPU_KERNEL", kernel)
    bounds = channel_boundaries(p, 200000)
    c, kmax = bounds[which]
    k = kmax + past
    plan = ff.fgemm_plan(1, 1, k, p)
    assert plan["channels"] == c + past
    h = p // 2
    M = 1
    for mc in plan["moduli"]:
        M *= mc
    X = k * h * h
    assert X <= M // 4
    if past == 0:
        assert X >= 0.75 * (M // 4), (X, M // 4)
    m, n = 288, 272
    rng = W.rng_for("worstcase", 3, p, k)
    A, B, C, s, t = W.sign_pattern_problem(rng, m, n, k, p, h, h)
    alpha, beta = int(rng.integers(1, p)), int(rng.integers(0, p))
    got = run(A, B, C, p, alpha, beta)
    assert np.array_equal(got, closed_form(s, t, k, h, h, p, alpha, beta, C))
    check_sampled(A, B, C, got, p, alpha, beta, seed=k)
    if k < 1000:
        assert np.array_equal(got, oracle.fgemm(A, B, p, alpha, beta, C))


# A shape whose last wave the CTA-pair kernel cuts along the inner dimension on
# a GB300 (74 resident pairs): 10 x 8 = 80 tiles of 256 x 256, ragged edges, so
# 6 tiles in the last wave, each in min(74 / 6, chunks, 4) parts.
STREAM_K_MN = (2523, 2043)


@pytest.mark.parametrize("p", [65521, 8388593, 2147483647])
def test_cut_last_wave_at_the_accumulator_bound(p, monkeypatch):
    """80 tiles on 74 pairs with four chunks per tile: each last-wave tile is
    cut into four parts, and the head adds three tails' residues to a full
    chunk at the accumulator bound (sign-pattern inputs, residues
    +-(m_c - 1)/2).  Every entry against the closed form, sampled entries
    against the oracle, and the whole result against the round-robin
    schedule (FFGPU_STREAMK=0)."""
    monkeypatch.setenv("FFGPU_KERNEL", "pair")
    m, n = STREAM_K_MN
    chunk = ff.fgemm_plan(m, n, 4096, p)["k_chunk"]
    k = 3 * chunk + 300
    plan = ff.fgemm_plan(m, n, k, p)
    assert plan["channels"] % 2 == 0 and plan["mode"] == 2
    x, used = largest_x_with_half_residues(p, plan["moduli"])
    rng = W.rng_for("worstcase", 2, p)
    A, B, C, s, t = W.sign_pattern_problem(rng, m, n, k, p, x, x)
    alpha, beta = int(rng.integers(1, p)), int(rng.integers(1, p))
    got = run(A, B, C, p, alpha, beta)
    assert np.array_equal(got, closed_form(s, t, k, x, x, p, alpha, beta, C))
    check_sampled(A, B, C, got, p, alpha, beta, seed=p % 1000)
    monkeypatch.setenv("FFGPU_STREAMK", "0")
    assert np.array_equal(run(A, B, C, p, alpha, beta), got)


@pytest.mark.parametrize("k", [2048, 3000])
def test_cut_last_wave_uniform_words(k, monkeypatch):
    """Uniform words (not reduced mod p) at the same shape with two and three
    chunks per tile (two and three parts): sampled entries against the
    oracle, Freivalds' test, and the round-robin schedule's result."""
    monkeypatch.setenv("FFGPU_KERNEL", "pair")
    p = 2147483647
    m, n = STREAM_K_MN
    rng = W.rng_for("square", 12, k)
    A, B, C = W.uniform_words(rng, (m, k)), W.uniform_words(rng, (k, n)), W.uniform_words(rng, (m, n))
    alpha, beta = int(rng.integers(0, p)), int(rng.integers(0, p))
    got = run(A, B, C, p, alpha, beta)
    check_sampled(A, B, C, got, p, alpha, beta, seed=k, count=2048)
    assert oracle.freivalds(A, B, C, got, p, alpha, beta, trials=2)
    monkeypatch.setenv("FFGPU_STREAMK", "0")
    assert np.array_equal(run(A, B, C, p, alpha, beta), got)


@pytest.mark.parametrize("p", [65521, 2147483647])
def test_cut_small_problem_at_the_accumulator_bound(p, monkeypatch):
    """Fewer tiles than resident pairs (1000 x 1000: 16 pair tiles), so the
    whole problem is one wave cut into four parts of about 17 k-steps: each
    part's first chunk is a full one at the accumulator bound (sign-pattern
    inputs, residues +-(m_c - 1)/2), and the head adds three tails' residues
    to it.  Every entry against the closed form, sampled entries against the
    oracle, the whole result against the round-robin schedule."""
    monkeypatch.setenv("FFGPU_KERNEL", "pair")
    m = n = 1000
    chunk = ff.fgemm_plan(m, n, 4096, p)["k_chunk"]
    k = 4 * chunk + 300
    plan = ff.fgemm_plan(m, n, k, p)
    assert plan["channels"] % 2 == 0 and plan["mode"] == 2
    x, used = largest_x_with_half_residues(p, plan["moduli"])
    rng = W.rng_for("worstcase", 3, p)
    A, B, C, s, t = W.sign_pattern_problem(rng, m, n, k, p, x, x)
    alpha, beta = int(rng.integers(1, p)), int(rng.integers(1, p))
    got = run(A, B, C, p, alpha, beta)
    assert np.array_equal(got, closed_form(s, t, k, x, x, p, alpha, beta, C))
    check_sampled(A, B, C, got, p, alpha, beta, seed=p % 997)
    monkeypatch.setenv("FFGPU_STREAMK", "0")
    assert np.array_equal(run(A, B, C, p, alpha, beta), got)


@pytest.mark.parametrize("m,k,n", [(1000, 2048, 1000), (700, 3000, 1100), (520, 2047, 300), (300, 4100, 1500)])
def test_cut_small_problems_uniform_words(m, k, n, monkeypatch):
    """Problems with fewer tiles than pairs, cut into two to four parts of at
    least a chunk of k-steps each (parts not aligned to chunks, ragged k and
    ragged tiles), against the oracle element by element."""
    monkeypatch.setenv("FFGPU_KERNEL", "pair")
    p = 2147483647
    rng = W.rng_for("square", 13, m, k, n)
    A, B, C = W.uniform_words(rng, (m, k)), W.uniform_words(rng, (k, n)), W.uniform_words(rng, (m, n))
    alpha, beta = int(rng.integers(0, p)), int(rng.integers(0, p))
    check(A, B, C, p, alpha, beta)
