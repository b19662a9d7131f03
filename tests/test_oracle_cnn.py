"""Pins of the CPU network reference: finite differences, a dense-matrix form
of the circular 3x3 convolution, and bfloat16 rounding."""
import numpy as np

from oracle import cnn


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 0.0])
    # 8 significand bits: 1 + 2^-8 is a tie -> even (1.0); 1 + 3*2^-8 -> 1 + 2^-6
    want = np.array([1.0, 1.0, 1.0 + 2 ** -7, 1.0 + 2 ** -6, -2.5, 0.0])
    np.testing.assert_array_equal(cnn.bf16_round(vals), want)


def test_conv_equals_dense_circular_matrix():
    rng = np.random.default_rng(0)
    H, Wd, ci, co = 5, 4, 3, 2
    a = rng.standard_normal((1, H, Wd, ci))
    W = rng.standard_normal((9, co, ci))
    b = rng.standard_normal(co)
    y = cnn.conv(a, W, b)
    for yy in range(H):
        for xx in range(Wd):
            for o in range(co):
                s = b[o]
                for t, (dy, dx) in enumerate(cnn.TAPS):
                    s += W[t, o] @ a[0, (yy + dy) % H, (xx + dx) % Wd]
                assert abs(y[0, yy, xx, o] - s) < 1e-12


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    chans = [4, 5, 5, 2]
    Ws, bs = cnn.init(chans, seed=2)
    bs = [rng.standard_normal(b.shape) * 0.1 for b in bs]
    x = rng.standard_normal((2, 6, 5, 4))
    tgt = rng.standard_normal((2, 6, 5, 2))

    def loss(Ws_, bs_, x_):
        acts, _ = cnn.forward(x_, Ws_, bs_)
        return 0.5 * np.sum((acts[-1] - tgt) ** 2)

    acts, pres = cnn.forward(x, Ws, bs)
    dWs, dbs, dx = cnn.backward(acts, pres, Ws, acts[-1] - tgt)
    h = 1e-6
    for l in range(len(Ws)):
        for idx in [(0, 0, 0), (4, 1, 2), (8, -1, -1)]:
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[l][idx] += h
            Wm[l][idx] -= h
            fd = (loss(Wp, bs, x) - loss(Wm, bs, x)) / (2 * h)
            assert abs(fd - dWs[l][idx]) < 1e-6 * max(1.0, abs(fd))
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[l][0] += h
        bm[l][0] -= h
        fd = (loss(Ws, bp, x) - loss(Ws, bm, x)) / (2 * h)
        assert abs(fd - dbs[l][0]) < 1e-6 * max(1.0, abs(fd))
    xp, xm = x.copy(), x.copy()
    xp[1, 3, 2, 1] += h
    xm[1, 3, 2, 1] -= h
    fd = (loss(Ws, bs, xp) - loss(Ws, bs, xm)) / (2 * h)
    assert abs(fd - dx[1, 3, 2, 1]) < 1e-6 * max(1.0, abs(fd))
