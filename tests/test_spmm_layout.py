"""The batched FP32 apply's shared-memory plan (iga_apply_f32_layout, the
numbers the kernel launches with) checked on the CPU: a model of the kernel's
per-thread index arithmetic (csrc/spmm.cu: 224 stage-1 threads, 288 stage-2
threads in half-warps) runs on those strides and must stay inside the
reported allocation, keep its vector accesses aligned, write every output
once, and reproduce y = (Y2 (x) X1 + Z2 (x) W1) x.  Covers every order the
kernel is compiled for (p = 2..8), both grid layouts and ragged grids."""
import numpy as np
import pytest

G1, G2 = 224, 288          # threads of the two warp groups (spmm.cu kG1, kG2)


@pytest.fixture(scope="module")
def B():
    from paper_2107_05337_gb300 import binding, build
    build.build()
    return binding


def _band(n, p, rng):
    W = 2 * p + 1
    b = rng.standard_normal((n, W))
    for i in range(n):
        for o in range(W):
            if not 0 <= i - p + o < n:
                b[i, o] = 0.0
    return b


def _dense(b, p):
    n, W = b.shape
    A = np.zeros((n, n))
    for i in range(n):
        for o in range(W):
            if 0 <= i - p + o < n:
                A[i, i - p + o] = b[i, o]
    return A


def _model(lay, n, p, X1, W1, Y2, Z2, x):
    """One column through the kernel's indexing; returns y and asserts bounds."""
    W = 2 * p + 1
    J, xs, ns, R, nb = lay["J"], lay["xs"], lay["ns"], lay["rows"], lay["ring"]
    V = (J + W - 1 + J - 1) // J
    G = (n + J - 1) // J
    slot = n * xs
    buf = 2 * R * ns
    total = nb * slot + 2 * buf
    assert 4 * total == lay["smem"]
    sm = np.zeros(total)
    s, kb = nb - 1, 1                          # last ring slot, second (tm, tk) buffer
    # copies: warp w rows w, w + 7, ...; lane columns lane, lane + 32, lane + 64
    for t in range(G1):
        wq, lane = t >> 5, t & 31
        for iy in range(wq, n, G1 // 32):
            for m in range(3):
                if lane + 32 * m < n:
                    e = s * slot + iy * xs + p + lane + 32 * m
                    assert s * slot <= e < (s + 1) * slot
                    sm[e] = x[iy * n + lane + 32 * m]
    # stage 1: thread (g, r0) owns grid columns J g .. J g + J - 1 of rows r0, r0 + R1, ...
    R1 = G1 // G
    tb = nb * slot + kb * buf
    for t in range(G1):
        g, r0 = t % G, t // G
        if r0 >= R1:
            continue
        cols = [J * g + j for j in range(J)]
        a = np.array([[X1[c, o] if c < n else 0.0 for o in range(W)] for c in cols])
        b = np.array([[W1[c, o] if c < n else 0.0 for o in range(W)] for c in cols])
        for iy in range(r0, n, R1):
            r = s * slot + iy * xs + J * g
            assert r % J == 0 and r + J * V <= (s + 1) * slot
            v = sm[r:r + J * V]
            d = tb + 2 * ((p + iy) * ns + J * g)
            assert d % 4 == 0 and d + 2 * J <= tb + buf
            for j in range(J):
                sm[d + 2 * j] = a[j] @ v[j:j + W]
                sm[d + 2 * j + 1] = b[j] @ v[j:j + W]
    # stage 2: half-warp h row groups h, h + 18, ...; lane c columns c, c + 16, ...
    y = np.full(n * n, np.nan)
    hits = np.zeros(n * n, dtype=int)
    for u in range(G2):
        h, c = u >> 4, u & 15
        for gy in range(h, G, G2 // 16):
            rows = [J * gy + j for j in range(J)]
            cy = np.array([[Y2[r, o] if r < n else 0.0 for o in range(W)] for r in rows])
            cz = np.array([[Z2[r, o] if r < n else 0.0 for o in range(W)] for r in rows])
            for ix in range(c, n, 16):
                idx = [tb + 2 * ((J * gy + q) * ns + ix) for q in range(J + W - 1)]
                assert min(idx) >= tb and max(idx) + 1 < tb + buf and idx[0] % 2 == 0
                um, uk = sm[idx], sm[[i + 1 for i in idx]]
                for j in range(J):
                    if J * gy + j < n:
                        y[(J * gy + j) * n + ix] = cy[j] @ um[j:j + W] + cz[j] @ uk[j:j + W]
                        hits[(J * gy + j) * n + ix] += 1
    assert (hits == 1).all()
    return y


@pytest.mark.parametrize("n,p", [(16, 2), (65, 3), (66, 4), (26, 4), (67, 5), (11, 5), (68, 6),
                                 (40, 7), (69, 7), (80, 8), (84, 4), (13, 3)])
def test_layout_model_in_bounds_and_exact(B, n, p):
    lay = B.apply_f32_layout(n, p)
    assert lay["cap"] in (68, 84) and lay["ring"] >= 2
    rng = np.random.default_rng(n * 10 + p)
    X1, W1, Y2, Z2 = (_band(n, p, rng) for _ in range(4))
    x = rng.standard_normal(n * n)
    want = (np.kron(_dense(Y2, p), _dense(X1, p)) + np.kron(_dense(Z2, p), _dense(W1, p))) @ x
    y = _model(lay, n, p, X1, W1, Y2, Z2, x)
    assert np.abs(y - want).max() <= 1e-12 * np.abs(want).max()


def test_grids_beyond_the_layouts_are_refused(B):
    assert B.apply_f32_layout(85, 4)["cap"] == 0
    assert B.apply_f32_layout(66, 4, smem_max=64 * 1024)["cap"] == 0
    with pytest.raises(B.IgmError):
        B.apply_f32_layout(66, 9)
