"""The index maps of the DCT column kernels on the 6-stage engine, checked
on the CPU against the definitions they implement (no GPU, no kernel run).

The kernels hold, after their last stage group, the complex DFT Z of the
reordered line (Makhoul's reduction of the DCT-II, Section 5's "similar
transforms"), spread over threads and CTAs: thread (lo, w) of a CTA holds
Z[k + 4096 t] at k = lo + 64 r for the register indices r it kept.  Each
output X[K] needs Z[K] and Z[N - K] (two real columns per complex line, the
"two for one" split).  These tests rebuild the kernels' hand-over slots,
pairings, rotations and staged output rows in numpy from a random Z and
check every output row against the two-for-one formula, written once:
  - the L2-exchange cluster kernel (col_dct_pack_l2_kernel, pair and four
    CTAs): blocks t >= CS/2 go to CTA CS-1-q, rows 0 as special cases;
  - the single-CTA forward kernel (col_dct_tma64_kernel): values r >= 32
    handed to thread 64 - lo through shared memory;
  - the single-CTA inverse kernel (col_idct_tma64_kernel): the pre-rotation
    of the scrambled gather and the even / odd output rows.
"""
import numpy as np
import pytest

L, NL, S0, KW, W, T, R = 12, 4096, 6, 2, 4, 256, 64


def brev(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2)


def dct_pair(zk, zp, cs):
    """Outputs at k and N-k of the two real lines of a complex line."""
    c, s = cs.real * 0.5, cs.imag * 0.5
    sr, dr = zk.real + zp.real, zp.real - zk.real
    si, di = zk.imag + zp.imag, zk.imag - zp.imag
    return complex(c * sr + s * di, c * si + s * dr), complex(s * sr - c * di, s * si - c * dr)


def two_for_one(Z):
    """(X_a + i X_b)[k] for z = v_a + i v_b, Z = DFT(z): the DCT-II outputs of
    both real lines from X[k] = Re(exp(-i pi k / (2N)) V[k])."""
    N = Z.shape[0]
    k = np.arange(N)
    kp = (-k) % N
    Va = (Z + np.conj(Z[kp])) / 2
    Vb = (Z - np.conj(Z[kp])) / 2j
    rot = np.exp(-1j * np.pi * k / (2 * N))[:, None]
    return (rot * Va).real + 1j * (rot * Vb).real


@pytest.mark.parametrize("CL", [1, 2])
def test_cluster_mirror_exchange_covers_every_row(CL):
    CS, HT = 1 << CL, (1 << CL) // 2
    NN = NL << CL
    KR, OUT = R >> CL, NL >> CL
    rng = np.random.default_rng(CL)
    Z = rng.standard_normal((NN, W)) + 1j * rng.standard_normal((NN, W))
    post = np.exp(1j * np.pi * np.arange(NN // 2 + 1) / (2 * NN))

    def kbase(q):
        return sum(((q >> j) & 1) * ((R >> j) // 2) for j in range(CL)) << S0

    a = {}
    for q in range(CS):
        for tid in range(T):
            lo, w = tid >> KW, tid & 3
            for t in range(CS):
                for i in range(KR):
                    a[q, tid, t * KR + i] = Z[(t << L) + kbase(q) + ((i << S0) | lo), w]
    # the exchange: blocks t >= HT to CTA CS-1-q, rows 0 of CTAs 2 and 3 of
    # four to each other
    MREG = HT * KR * T
    slot = np.full(CS * MREG, np.nan + 0j)
    writes = np.zeros(CS * MREG, int)
    for q in range(CS):
        for tid in range(T):
            lo, w = tid >> KW, tid & 3
            tid_r = ((((1 << S0) - lo) & ((1 << S0) - 1)) << KW) | w
            for t in range(HT, CS):
                for i in range(KR):
                    if lo == 0 and i == 0:
                        continue
                    i_r = KR - 1 - i if lo else KR - i
                    j = (CS - 1 - q) * MREG + ((CS - 1 - t) * KR + i_r) * T + tid_r
                    slot[j], writes[j] = a[q, tid, t * KR + i], writes[j] + 1
            if CL == 2 and q >= 2 and lo == 0:
                for t in range(HT, CS):
                    j = (q ^ 1) * MREG + (CS - 1 - t) * KR * T + w
                    slot[j], writes[j] = a[q, tid, t * KR], writes[j] + 1
    assert writes.max() == 1
    out = np.full((NN, W), np.nan + 0j)
    count = np.zeros((NN, W), int)
    for q in range(CS):
        kb = kbase(q)
        own = np.full((HT * OUT, W), np.nan + 0j)
        rev = np.full((HT * OUT, W), np.nan + 0j)
        for tid in range(T):
            lo, w = tid >> KW, tid & 3
            r0 = [a[q, tid, t * KR] for t in range(CS)]
            if q == 0 and lo == 0:   # K = N/2 pairs with itself
                out[NN // 2, w] = dct_pair(r0[HT], r0[HT], post[NN // 2])[0]
                count[NN // 2, w] += 1
            rot_lo = post[lo]
            for t in range(HT):
                for i in range(KR):
                    row = (i << S0) | lo
                    zk = a[q, tid, t * KR + i]
                    if i == 0 and lo == 0 and q == 0:
                        zp = zk if t == 0 else r0[CS - t]
                    elif i == 0 and lo == 0 and kb == NL // 2:
                        zp = r0[CS - 1 - t]
                    else:
                        j = q * MREG + (t * KR + i) * T + tid
                        assert writes[j] == 1
                        zp = slot[j]
                    cs = post[(t << L) + kb + (i << S0)] * rot_lo   # shared block start x own factor
                    xk, xp = dct_pair(zk, zp, cs)
                    own[t * OUT + row, w] = xk
                    rev[t * OUT + OUT - 1 - row, w] = xp
        for t in range(HT):
            y = (t << L) + kb
            assert y % 256 == 0                      # whole 256-row boxes
            out[y:y + OUT] = own[t * OUT:(t + 1) * OUT]
            count[y:y + OUT] += 1
            y0 = NN - (t << L) - kb - OUT + 1        # reversed range, any row
            assert y0 > 0
            for s in range(OUT):
                if y0 + s < NN:                      # the row past the image is not stored
                    out[y0 + s] = rev[t * OUT + s]
                    count[y0 + s] += 1
    assert count.min() == 1 and count.max() == 1
    want = two_for_one(Z)
    assert np.abs(out - want).max() <= 1e-12 * np.abs(want).max()


def test_single_cta_forward_hand_over():
    N, HALF = NL, NL // 2
    rng = np.random.default_rng(3)
    Z = rng.standard_normal((N, W)) + 1j * rng.standard_normal((N, W))
    post = np.exp(1j * np.pi * np.arange(HALF + 1) / (2 * N))
    a = np.array([[Z[(tid >> KW) + 64 * r, tid & 3] for r in range(R)] for tid in range(T)])
    stage = np.full(HALF * W, np.nan + 0j)
    writes = np.zeros(HALF * W, int)
    for tid in range(T):                       # values r >= 32 to thread 64 - lo
        lo, w = tid >> KW, tid & 3
        if lo:
            tid_r = (((1 << S0) - lo) << KW) | w
            for r in range(R // 2, R):
                j = (R - 1 - r) * T + tid_r
                stage[j], writes[j] = a[tid, r], writes[j] + 1
    assert writes.max() == 1
    fill1 = np.full((HALF, W), np.nan + 0j)
    fill2 = np.full((HALF, W), np.nan + 0j)
    for tid in range(T):
        lo, w = tid >> KW, tid & 3
        b = a[tid].copy()
        if lo == 0:                            # k = N/2 pairs with itself
            fill2[0, w] = dct_pair(b[R // 2], b[R // 2], post[HALF])[0]
        for r in range(R // 2):
            zk = b[r]
            if lo:
                assert writes[r * T + tid] == 1
                zp = stage[r * T + tid]
            else:
                zp = zk if r == 0 else b[R - r]
            xk, xp = dct_pair(zk, zp, post[64 * r] * post[lo])
            b[r] = xk
            b[R // 2 if r == 0 else R - r] = xp
        for r in range(R // 2):
            k = (r << S0) | lo
            fill1[k, w] = b[r]
            if lo or r:
                fill2[HALF - k, w] = b[R // 2 if r == 0 else R - r]
    out = np.concatenate([fill1, fill2])
    assert not np.isnan(out).any()
    want = two_for_one(Z)
    assert np.abs(out - want).max() <= 1e-12 * np.abs(want).max()


def test_single_cta_inverse_gather_and_rows():
    """Pre-rotation of the scrambled gather (64 shared block starts times a
    per-thread factor), then x[2n] = v[n], x[2n+1] = v[N-1-n]; the result is
    the DCT-III of both real columns, x = (1/N)(X0 + 2 sum X[k] cos(..))."""
    N, HALF, G, HB = NL, NL // 2, 6, 6
    rng = np.random.default_rng(5)
    X = rng.standard_normal((N, W)) + 1j * rng.standard_normal((N, W))
    post = np.exp(1j * np.pi * np.arange(HALF + 1) / (2 * N))
    rot_top = []
    for j in range(R):
        top = brev(j, G) << HB
        p = post[top if top <= HALF else N - top]
        rot_top.append(p if top <= HALF else complex(p.imag, p.real))
    Zs = np.zeros((N, W), complex)
    seen = np.zeros((N, W), int)
    for tid in range(T):
        w, hib = tid & 3, (tid >> KW) & 63
        for r in range(R):
            k = (brev(r, G) << HB) | hib
            xn = X[k, w]
            xm = X[(N - k) & (N - 1), w] if k else 0j
            cs = rot_top[r] * post[hib]
            c, s = cs.real, cs.imag
            Zs[k, w] = complex(c * xn.real + s * xm.real - s * xn.imag + c * xm.imag,
                               s * xn.real - c * xm.real + c * xn.imag + s * xm.imag)
            seen[k, w] += 1
    assert seen.min() == 1 and seen.max() == 1
    v = np.fft.ifft(Zs, axis=0)                # the inverse DFT times the scale 1/N
    out = np.full((N, W), np.nan + 0j)
    for tid in range(T):
        w, lo = tid & 3, (tid >> KW) & 63
        for r in range(R):
            k = (r << S0) | lo
            if r < R // 2:
                out[2 * k, w] = v[k, w]
            else:
                out[2 * (N - 1 - k) + 1, w] = v[k, w]
    assert not np.isnan(out).any()
    rows = np.sort(rng.choice(N, 64, replace=False))    # sampled output rows
    k = np.arange(N)[None, :]
    wts = np.where(np.arange(N) == 0, 1.0, 2.0)
    C = np.cos(np.pi * k * (2 * rows[:, None] + 1) / (2 * N)) * wts / N
    want = C @ X.real + 1j * (C @ X.imag)
    assert np.abs(out[rows] - want).max() <= 1e-11 * np.abs(want).max()
