"""Host model of the single-precision group FFT's data movement (fft_kernels.cu:
group_fft, tile_ffts, spread_tasks): a pencil of N = F Q points on Q lanes
with F values each, n = q + Q m, k = k1 + F k2.

The model follows the kernel's steps lane by lane (F-point DFT over m in
registers, twiddle W_N^(q k1), exchange through slot k1 Q + (q' ^ (k1 mod Q)),
Q-point DFTs over q' for k1 = q + Q r) and checks that
  * the result is the DFT (numpy), forward and inverse, for every N;
  * the exchange writes every slot exactly once (a permutation);
  * within a group, the exchange's stores (fixed k1) and loads (fixed r, q')
    fall on distinct 8-byte banks;
  * the task layout p = t + T g covers every pencil once.
"""
import numpy as np
import pytest

SHAPES = {32: (8, 4), 64: (8, 8), 128: (16, 8), 256: (16, 16)}


def _radix2(v, direction):
    """Natural-order DFT by radix-2 decimation in time (the register DFT)."""
    n = len(v)
    lg = n.bit_length() - 1
    a = [v[int(format(i, f"0{lg}b")[::-1], 2)] for i in range(n)] if lg else list(v)
    h = 1
    while h < n:
        for g in range(0, n, 2 * h):
            for k in range(h):
                b = a[g + k + h] * np.exp(direction * 2j * np.pi * k / (2 * h))
                u = a[g + k]
                a[g + k], a[g + k + h] = u + b, u - b
        h *= 2
    return a


def _group_fft(x, F, Q, direction):
    N = F * Q
    R = F // Q
    regs = {}
    for q in range(Q):
        v = _radix2([x[q + Q * m] for m in range(F)], direction)
        regs[q] = [v[k1] * np.exp(direction * 2j * np.pi * ((q * k1) % N) / N) for k1 in range(F)]
    slots = [None] * N
    for q in range(Q):
        for k1 in range(F):
            j = k1 * Q + (q ^ (k1 & (Q - 1)))
            assert slots[j] is None
            slots[j] = regs[q][k1]
    assert all(s is not None for s in slots)
    out = [None] * N
    for q in range(Q):
        for r in range(R):
            w = _radix2([slots[(q + Q * r) * Q + (i ^ q)] for i in range(Q)], direction)
            for k2 in range(Q):
                k = q + Q * r + F * k2
                assert out[k] is None
                out[k] = w[k2]
    return np.array(out)


@pytest.mark.parametrize("N", sorted(SHAPES))
@pytest.mark.parametrize("direction", [-1, 1])
def test_group_fft_is_the_dft(N, direction):
    F, Q = SHAPES[N]
    rng = np.random.default_rng(N)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    got = _group_fft(x, F, Q, direction)
    ref = np.fft.fft(x) if direction < 0 else np.fft.ifft(x) * N
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("N", sorted(SHAPES))
def test_exchange_is_bank_conflict_free_within_a_group(N):
    F, Q = SHAPES[N]
    # 8-byte entries: 16 banks of 8 bytes; a group's Q lanes see contiguous slots
    for k1 in range(F):
        banks = [(k1 * Q + (q ^ (k1 & (Q - 1)))) % 16 for q in range(Q)]
        assert len(set(banks)) == Q
    for r in range(F // Q):
        for i in range(Q):
            banks = [((q + Q * r) * Q + (i ^ q)) % 16 for q in range(Q)]
            assert len(set(banks)) == Q


@pytest.mark.parametrize("G", [2, 4, 8])
def test_task_layout_covers_every_pencil_once(G):
    MOD, RES = 32 // G, 16 // G
    for P in range(1, 300):
        nt = (P + G - 1) // G
        if G > 2:
            nt += ((RES - nt) % MOD + MOD) % MOD
        pencils = [t + nt * g for t in range(nt) for g in range(G)]
        assert len(set(pencils)) == len(pencils)
        assert set(range(P)) <= set(pencils)
