"""The row-strip and curved forms of the batched FP32 apply, checked on the CPU
through their launch plans (iga_apply_f32_plan, the numbers the kernels launch
with): a model of each kernel's index arithmetic (csrc/spmm.cu
k_spmm32_strip, k_spmm32_curved) runs on the plan, over every CTA of the
grid, and must keep every shared-memory and global access inside its
allocation, write every output exactly once, and reproduce the dense product
(Sec. 2: y = (Y2 (x) X1 + Z2 (x) W1) x on the unit square; an assembled
(2p+1)^2 stencil per grid point on a curved map).  Covers every order the
kernels are compiled for (p = 2..8), ragged strips and tiles, and grids up to
the largest a descriptor allows; the GPU parity tests cover p = 2..6."""
import numpy as np
import pytest

SMEM_MAX = 232448           # opt-in shared memory per block of the GB300
SMS = 152


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


def _strip_model(plan, n, p, M1, K1, cf, X, strips=None):
    """Every CTA (strip s, column group g) of the launch on columns X [nrhs, n*n]:
    returns Y (NaN where nothing was written) and the write counts."""
    W = 2 * p + 1
    SR, T, smem, nstrips, groups = (plan[k] for k in ("SR", "threads", "smem", "strips", "groups"))
    RS, XW = SR + 2 * p, n + 2 * p
    STAGE = RS * XW
    assert 4 * (2 * SR * W + 2 * STAGE) == smem <= SMEM_MAX
    assert T % 32 == 0 and 32 <= T <= 512 and nstrips == -(-n // SR)
    nrhs, N = X.shape
    xm, xk, wm, wk, ym, yk, zm, zk = cf
    Y = np.full((nrhs, N), np.nan)
    writes = np.zeros((nrhs, N), dtype=np.int64)
    for s in (range(nstrips) if strips is None else strips):
        r0 = s * SR
        rows = min(SR, n - r0)
        assert rows >= 1
        # (Y2, Z2) of the strip's rows (clamped rows past the grid are never used)
        iyc = np.minimum(r0 + np.arange(SR), n - 1)
        c2y = yk * K1[iyc] + ym * M1[iyc]
        c2z = zk * K1[iyc] + zm * M1[iyc]
        for g in range(groups):
            for b in range(g, nrhs, groups):
                # staging: staged row q, column c <- x[r0 - p + q][c - p], zero outside
                q = np.arange(RS)[:, None]
                c = np.arange(XW)[None, :]
                iy, ix = r0 - p + q, c - p
                on = (iy >= 0) & (iy < n) & (ix >= 0) & (ix < n)
                gi = iy * n + ix
                assert gi[on].min() >= 0 and gi[on].max() < N
                xs = np.where(on, X[b][np.clip(gi, 0, N - 1)], 0.0).reshape(-1)
                for ix0 in range(0, n, T):
                    t = np.arange(T)
                    mine = ix0 + t < n
                    ixc = np.minimum(ix0 + t, n - 1)
                    a1x = xk * K1[ixc] + xm * M1[ixc]
                    a1w = wk * K1[ixc] + wm * M1[ixc]
                    win = [None] * W
                    for q0 in range(0, RS, W):
                        for k in range(W):
                            qq = q0 + k
                            if qq >= RS:
                                continue
                            idx = qq * XW + ixc[:, None] + np.arange(W)[None, :]
                            assert idx.min() >= 0 and idx.max() < STAGE
                            xr = xs[idx]
                            win[k] = (qq, (a1x * xr).sum(1), (a1w * xr).sum(1))
                            j = qq - 2 * p
                            if 0 <= j < rows:
                                acc = np.zeros(T)
                                for o in range(W):
                                    rq, tm, tk = win[(k + 1 + o) % W]
                                    assert rq == j + o      # the window holds staged row j + o
                                    acc += c2y[j, o] * tm + c2z[j, o] * tk
                                out = (r0 + j) * n + ixc[mine]
                                assert out.max() < N
                                Y[b, out] = acc[mine]
                                writes[b, out] += 1
    return Y, writes


CF = {"M": (1, 0, 0, 0, 1, 0, 0, 0), "K": (1, 0, 0, 1, 0, 1, 1, 0)}


@pytest.mark.parametrize("p", range(2, 9))
@pytest.mark.parametrize("n,nrhs", [(85, 3), (131, 7), (200, 2)])
def test_strip_model_every_order(B, p, n, nrhs):
    rng = np.random.default_rng(100 * p + n)
    M1, K1 = _band(n, p, rng), _band(n, p, rng)
    c = 0.37
    cf = (1, 0, 0, 1, 1, c, c, 0)           # M + c K, as iga_apply_f32 forms it
    plan = B.apply_f32_plan("strip", n, p, nrhs, SMS, SMEM_MAX)
    assert plan["SR"] >= 1
    X = rng.standard_normal((nrhs, n * n))
    Y, writes = _strip_model(plan, n, p, M1, K1, cf, X)
    assert np.all(writes == 1)
    Md, Kd = _dense(M1, p), _dense(K1, p)
    # (A_eta (x) A_xi) x on the row-major grid is A_eta X A_xi^T
    kron = lambda Ae, Ax, x: (Ae @ x.reshape(n, n) @ Ax.T).reshape(-1)
    want = np.array([kron(Md + c * Kd, Md, x) + kron(c * Md, Kd, x) for x in X])
    assert np.allclose(Y, want, rtol=1e-12, atol=1e-12)
    for which in ("M", "K"):
        Y, _ = _strip_model(plan, n, p, M1, K1, CF[which], X[:1])
        want = (kron(Md, Md, X[0]) if which == "M" else
                kron(Kd, Md, X[0]) + kron(Md, Kd, X[0]))
        assert np.allclose(Y[0], want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("p,n", [(2, 1024), (5, 1027), (8, 1030), (3, 513)])
def test_strip_model_largest_grids(B, p, n):
    """The largest grids (more grid columns than threads per CTA): the plan fits,
    and the first, a middle and the last (ragged) strip write their rows exactly
    once with the right values; rows are checked against the dense 1D factors
    applied to the sampled rows only."""
    rng = np.random.default_rng(7 + p)
    M1, K1 = _band(n, p, rng), _band(n, p, rng)
    plan = B.apply_f32_plan("strip", n, p, 1, SMS, SMEM_MAX)
    assert plan["SR"] >= 1 and plan["threads"] == 512
    X = rng.standard_normal((1, n * n))
    last = plan["strips"] - 1
    Y, writes = _strip_model(plan, n, p, M1, K1, CF["K"], X, strips=[0, last // 2, last])
    Md, Kd = _dense(M1, p), _dense(K1, p)
    Xg = X[0].reshape(n, n)
    for s in (0, last // 2, last):
        r0, r1 = s * plan["SR"], min(n, (s + 1) * plan["SR"])
        want = Kd[r0:r1] @ Xg @ Md.T + Md[r0:r1] @ Xg @ Kd.T   # K = K1 (x) M1 + M1 (x) K1
        got = Y[0].reshape(n, n)[r0:r1]
        assert np.all(writes[0].reshape(n, n)[r0:r1] == 1)
        assert np.allclose(got, want, rtol=1e-11, atol=1e-11)


def _curved_model(plan, n, p, Aq, X, ld):
    """Every CTA (tile, column group) of the curved launch on X [nrhs, ld]:
    coefficient q of point i at Aq[q, i] (q = (dy + p)(2p + 1) + dx + p)."""
    W = 2 * p + 1
    TR, TC, HR, HC, tiles, groups = (plan[k] for k in ("TR", "TC", "HR", "HC", "tiles", "groups"))
    assert (HR, HC) == (TR + 2 * p, TC + 2 * p) and TR * 32 == 256 and TC == 32
    assert 2 * 16 * HR * HC <= SMEM_MAX
    tilesx = -(-n // TC)
    assert tiles == tilesx * -(-n // TR)
    nrhs = X.shape[0]
    N = n * n
    ngroups = -(-nrhs // 4)
    Y = np.full((nrhs, ld), np.nan)
    writes = np.zeros((nrhs, ld), dtype=np.int64)
    lane = np.arange(256) & 31
    wr = np.arange(256) >> 5
    for tile in range(tiles):
        ix0, iy0 = (tile % tilesx) * TC, (tile // tilesx) * TR
        ix, iy = ix0 + lane, iy0 + wr
        mine = (ix < n) & (iy < n)
        pt = np.where(mine, iy * n + ix, 0)
        v = Aq[:, pt]                                   # [Q, 256]: the thread's coefficients
        for gy in range(groups):
            for g in range(gy, ngroups, groups):
                # staging: element e -> column 4g + (e & 3) at staged point e >> 2
                e = np.arange(4 * HR * HC)
                b, pos = e & 3, e >> 2
                r, c = pos // HC, pos % HC
                jy, jx, col = iy0 - p + r, ix0 - p + c, 4 * g + b
                on = (jy >= 0) & (jy < n) & (jx >= 0) & (jx < n) & (col < nrhs)
                gi = col * ld + jy * n + jx
                assert gi[on].min() >= 0 and gi[on].max() < nrhs * ld
                src = X.reshape(-1)[np.clip(gi, 0, nrhs * ld - 1)]
                xs = np.where(on, src, 0.0).reshape(HR * HC, 4)
                acc = np.zeros((256, 4))
                for dy in range(W):
                    for dx in range(W):
                        k = wr * HC + lane + dy * HC + dx
                        assert k.max() < HR * HC
                        acc += v[dy * W + dx][:, None] * xs[k]
                for bb in range(4):
                    cc = 4 * g + bb
                    if cc < nrhs:
                        out = cc * ld + pt[mine]
                        Y[cc, pt[mine]] = acc[mine, bb]
                        writes[cc, pt[mine]] += 1
                        assert out.max() < nrhs * ld
    return Y[:, :N], writes[:, :N]


@pytest.mark.parametrize("p", range(2, 9))
@pytest.mark.parametrize("n,nrhs,pad", [(15, 5, 1), (40, 13, 0), (67, 2, 3)])
def test_curved_model_every_order(B, p, n, nrhs, pad):
    rng = np.random.default_rng(1000 + 10 * p + n)
    W = 2 * p + 1
    N = n * n
    Aq = rng.standard_normal((W * W, N))
    plan = B.apply_f32_plan("curved", n, p, nrhs, SMS, SMEM_MAX)
    X = rng.standard_normal((nrhs, N + pad))
    Y, writes = _curved_model(plan, n, p, Aq, X, N + pad)
    assert np.all(writes == 1)
    # y_i = sum over the stencil of point i of a_q x_(neighbour q), neighbours in the grid only
    Xg = X[:, :N].reshape(nrhs, n, n)
    want = np.zeros((nrhs, n, n))
    iy, ix = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for dy in range(W):
        for dx in range(W):
            jy, jx = iy + dy - p, ix + dx - p
            ok = (jy >= 0) & (jy < n) & (jx >= 0) & (jx < n)
            a = Aq[dy * W + dx].reshape(n, n)
            want += np.where(ok, a, 0.0) * Xg[:, np.clip(jy, 0, n - 1), np.clip(jx, 0, n - 1)]
    assert np.allclose(Y, want.reshape(nrhs, N), rtol=1e-12, atol=1e-12)


def test_plan_rejects_invalid_input(B):
    import ctypes
    out = (ctypes.c_int * 6)()
    for form, n, p, nrhs, sms, smem in [(0, 66, 4, 1, SMS, SMEM_MAX), (3, 66, 4, 1, SMS, SMEM_MAX),
                                        (1, 66, 9, 1, SMS, SMEM_MAX), (2, 0, 4, 1, SMS, SMEM_MAX),
                                        (1, 66, 4, -1, SMS, SMEM_MAX), (2, 66, 4, 1, 0, SMEM_MAX),
                                        (1, 66, 4, 1, SMS, 0)]:
        with pytest.raises(B.IgmError):
            B._check(B.lib().iga_apply_f32_plan(form, n, p, nrhs, sms, smem, out))
