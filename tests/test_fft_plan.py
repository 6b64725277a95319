"""Host-side checks of the index arithmetic of the register-resident FFT kernels
(csrc/fft_reg.cuh, csrc/fft.cuh, csrc/fft_stages.cuh), restated in NumPy. CPU only.

The kernels hold N = 2^LOGN complex values in T = N/8 threads, eight each, and move
them between radix-8 passes through shared memory. Checked here:

- the forward pass sequence is a DFT whose output element 8t + r holds the frequency
  that pos_of_freq places there, and the inverse sequence undoes it (times N);
- every mapping is bank-conflict free after the swizzle (16 lanes of a half-warp, one
  8-byte value each, hit 16 different bank pairs);
- each exchange writes exactly the addresses its thread read in the previous one, so
  consecutive exchanges need no barrier between them;
- split_freq is a bijection of the half spectrum 0..P/2.
"""
import numpy as np
import pytest


def elem(LOGN, p, t, r):
    NP8 = LOGN // 3
    if p >= NP8:
        return 8 * t + r
    lsr = LOGN - 3 * p - 3
    j = t & ((1 << lsr) - 1)
    g = t >> lsr
    return (g << (lsr + 3)) + j + (r << lsr)


def swz(i):
    return i ^ ((i >> 3) & 15)


def radices(LOGN):
    r = [3] * (LOGN // 3)
    if LOGN % 3:
        r.append(LOGN % 3)
    return r


def pos_of_freq(LOGN, k):
    p, kb, pb = 0, 0, LOGN
    for lr in radices(LOGN):
        digit = (k >> kb) & ((1 << lr) - 1)
        pb -= lr
        p |= digit << pb
        kb += lr
    return p


def dft(v, inv):
    R = len(v)
    w = np.exp((2j if inv else -2j) * np.pi * np.outer(np.arange(R), np.arange(R)) / R)
    return w @ v


def forward(x, LOGN):
    """The pass sequence of reg_fft_forward on one sequence; returns the values in MF
    order (element 8t + r) and the per-thread register arrays."""
    N, T = 1 << LOGN, 1 << (LOGN - 3)
    NP8, REM = LOGN // 3, LOGN % 3
    tw = np.exp(-2j * np.pi * np.arange(N) / N)
    v = np.array([[x[elem(LOGN, 0, t, r)] for r in range(8)] for t in range(T)])
    sm = np.zeros(N, complex)

    def exchange(pa, pb):
        for t in range(T):
            for r in range(8):
                sm[swz(elem(LOGN, pa, t, r))] = v[t, r]
        for t in range(T):
            for r in range(8):
                v[t, r] = sm[swz(elem(LOGN, pb, t, r))]

    for p in range(NP8):
        if p > 0:
            exchange(p - 1, p)
        lsr = LOGN - 3 * p - 3
        for t in range(T):
            v[t] = dft(v[t], False)
            step = (t & ((1 << lsr) - 1)) << (3 * p)
            for q in range(1, 8):
                v[t, q] *= tw[(q * step) % N]
    if REM:
        exchange(NP8 - 1, NP8)
        R = 1 << REM
        for t in range(T):
            for b in range(0, 8, R):
                v[t, b:b + R] = dft(v[t, b:b + R], False)
    return v.reshape(-1).copy(), v


def inverse(v, LOGN):
    N, T = 1 << LOGN, 1 << (LOGN - 3)
    NP8, REM = LOGN // 3, LOGN % 3
    tw = np.exp(-2j * np.pi * np.arange(N) / N)
    v = v.copy()
    sm = np.zeros(N, complex)

    def exchange(pa, pb):
        for t in range(T):
            for r in range(8):
                sm[swz(elem(LOGN, pa, t, r))] = v[t, r]
        for t in range(T):
            for r in range(8):
                v[t, r] = sm[swz(elem(LOGN, pb, t, r))]

    if REM:
        R = 1 << REM
        for t in range(T):
            for b in range(0, 8, R):
                v[t, b:b + R] = dft(v[t, b:b + R], True)
        exchange(NP8, NP8 - 1)
    for p in range(NP8 - 1, -1, -1):
        lsr = LOGN - 3 * p - 3
        for t in range(T):
            step = (t & ((1 << lsr) - 1)) << (3 * p)
            for q in range(1, 8):
                v[t, q] *= np.conj(tw[(q * step) % N])
            v[t] = dft(v[t], True)
        if p > 0:
            exchange(p, p - 1)
    out = np.zeros(N, complex)
    for t in range(T):
        for r in range(8):
            out[elem(LOGN, 0, t, r)] = v[t, r]
    return out


@pytest.mark.parametrize("LOGN", [7, 8, 9, 10, 11, 13])
def test_forward_is_a_dft_in_digit_reversed_order_and_inverse_undoes_it(LOGN):
    N = 1 << LOGN
    rng = np.random.default_rng(LOGN)
    x = rng.normal(size=N) + 1j * rng.normal(size=N)
    y, regs = forward(x, LOGN)
    X = np.fft.fft(x)
    pos = np.array([pos_of_freq(LOGN, k) for k in range(N)])
    assert sorted(pos) == list(range(N))
    assert np.allclose(y[pos], X, rtol=1e-10, atol=1e-9 * np.abs(X).max())
    assert np.allclose(inverse(regs, LOGN), N * x, atol=1e-9 * N * np.abs(x).max())


@pytest.mark.parametrize("LOGN", [7, 8, 9, 10, 11, 12, 13])
def test_swizzled_mappings_are_bank_conflict_free(LOGN):
    T = 1 << (LOGN - 3)
    for p in range(LOGN // 3 + 1):
        for r in range(8):
            for h0 in range(0, T, 16):
                banks = [swz(elem(LOGN, p, t, r)) % 16 for t in range(h0, min(h0 + 16, T))]
                assert len(set(banks)) == len(banks), (p, r, h0)


@pytest.mark.parametrize("LOGN", [7, 8, 9, 10, 11, 12, 13])
def test_mappings_are_permutations_and_swizzle_stays_in_block(LOGN):
    N, T = 1 << LOGN, 1 << (LOGN - 3)
    for p in range(LOGN // 3 + 1):
        e = sorted(elem(LOGN, p, t, r) for t in range(T) for r in range(8))
        assert e == list(range(N))
    assert all(swz(i) // 16 == i // 16 for i in range(N))


@pytest.mark.parametrize("LOGN", [7, 10, 11, 12, 13])
def test_each_exchange_writes_what_its_thread_read_last(LOGN):
    # forward exchanges read mapping p and the next one writes mapping p; the inverse
    # walks them backwards; so a thread only overwrites addresses it has read itself
    T = 1 << (LOGN - 3)
    NP8, REM = LOGN // 3, LOGN % 3
    last = NP8 if REM else NP8 - 1
    fwd = [(p - 1, p) for p in range(1, NP8)] + ([(NP8 - 1, NP8)] if REM else [])
    inv = [(b, a) for (a, b) in reversed(fwd)]
    seq = fwd + inv
    for (a0, b0), (a1, b1) in zip(seq, seq[1:]):
        assert a1 == b0
        for t in range(T):
            read = {swz(elem(LOGN, b0, t, r)) for r in range(8)}
            write = {swz(elem(LOGN, a1, t, r)) for r in range(8)}
            assert read == write
    assert seq[len(fwd) - 1][1] == last and seq[len(fwd)][0] == last


def split_warp(LOGP, j):
    """Lanes of a warp take frequencies P/64 apart."""
    H = 1 << (LOGP - 1)
    if j >= H:
        return j
    return (j & 31) * (H // 32) + (j >> 5)


def split_half(LOGP, j):
    """Lane l of each half-warp takes kx = l P/32 + j div 16."""
    H = 1 << (LOGP - 1)
    if j >= H:
        return j
    return (j & 15) * (H // 16) + (j >> 4)


def split_freq(LOGP, j):
    # the map the row kernels use at each FFT size
    return split_warp(LOGP, j) if LOGP in (9, 12) else split_half(LOGP, j)


@pytest.mark.parametrize("LOGP", [7, 8, 9, 10, 11, 12, 13])
def test_split_freq_is_a_bijection_of_the_half_spectrum(LOGP):
    H = 1 << (LOGP - 1)
    assert sorted(split_freq(LOGP, j) for j in range(H + 1)) == list(range(H + 1))


def split_wavefronts(mapf, LOGP):
    """Shared-memory wavefronts of the split pass of one row pair (three channels, the
    accesses at pos(kx) and at pos(P - kx)): per half-warp, the largest number of distinct
    8-byte words that share a bank pair."""
    P = 1 << LOGP
    NH = P // 2 + 1
    total = 0
    for c in range(3):
        for w0 in range(0, NH, 32):
            for mirror in (False, True):
                for half in (0, 16):
                    banks = {}
                    for lane in range(half, half + 16):
                        j = w0 + lane
                        if j >= NH:
                            continue
                        kx = mapf(LOGP, j)
                        q = (P - kx) % P if mirror else kx
                        a = c * P + swz(pos_of_freq(LOGP, q))
                        banks.setdefault(a % 16, set()).add(a)
                    total += max((len(v) for v in banks.values()), default=0)
    return total


@pytest.mark.parametrize("LOGP", [7, 8, 9, 10, 11, 12, 13])
def test_split_map_is_the_better_of_the_two_for_the_banks(LOGP):
    used = split_wavefronts(split_freq, LOGP)
    assert used <= min(split_wavefronts(split_warp, LOGP), split_wavefronts(split_half, LOGP))
    # within 2 % of the conflict-free count (two accesses per frequency, 16 per wavefront)
    # except at P = 512 and 4096, where neither map reaches it
    ideal = 3 * 2 * sum((min(32, (P := 1 << LOGP) // 2 + 1 - w0) + 15) // 16
                        for w0 in range(0, (1 << LOGP) // 2 + 1, 32))
    if LOGP not in (9, 12):
        assert used <= 1.02 * ideal + 6, (used, ideal)


def _kernel_constant(name):
    """An integer constexpr of csrc/fft_kernels.cu, read from the source."""
    import os
    import re
    path = os.path.join(os.path.dirname(__file__), "..", "paper_2303_03964_gb300", "csrc", "fft_kernels.cu")
    with open(path) as f:
        m = re.search(r"constexpr int %s = (\d+);" % name, f.read())
    assert m, name
    return int(m.group(1))


def _row_blocks(LOGP, pairs):
    """Rows per block of a row pass (fft_kernels.cu: RegGeom with RowsFwdGeom or
    RowsInvGeom, `pairs` row pairs per thread where T = 256) and whether the block
    accesses its output / input columns as 32-byte runs."""
    T = (1 << LOGP) // 8
    RG = 1 if T >= 256 else 256 // T
    seq = T > 512
    rp = pairs if (not seq and T == 256) else 1
    RB = RG * (1 if seq else rp)
    return 2 * RB, (not seq) and RB % 2 == 0


@pytest.mark.parametrize("LOGP", range(7, 14))
@pytest.mark.parametrize("which", ["kRowsFwdPairs", "kRowsInvPairs"])
def test_row_blocks_cover_the_grid_and_32_byte_runs_stay_aligned_and_inside(LOGP, which):
    # every row y < G_max is in some block; the rows a block touches end below ystride
    # (= G_max rounded up to 32), and where the pass moves 32 bytes per column, each run
    # starts 32-byte aligned: column base (c NH + kx) ystride and row base ybase + 2q
    # (q even), in float2 units of 8 bytes, from a 256-byte aligned array
    P = 1 << LOGP
    NH = P // 2 + 1
    rows, wide = _row_blocks(LOGP, _kernel_constant(which))
    for G_max in range(max(1, P // 4 - 40), P // 2 + 1):
        ystride = -(-G_max // 32) * 32
        blocks = -(-G_max // rows)
        assert blocks * rows >= G_max
        assert (blocks - 1) * rows + rows - 1 < ystride
        if wide:
            for blk in (0, 1, blocks - 1):
                ybase = blk * rows
                for q in range(0, rows // 2, 2):
                    for col in (0, 1, 3 * NH - 1):
                        assert 8 * (col * ystride + ybase + 2 * q) % 32 == 0
    # the spectrum rows 0..P/2 of the forward pass, into S1 with P rows per column
    blocks = -(-(P // 2 + 1) // rows)
    assert (blocks - 1) * rows + rows - 1 < P
