"""Pins of the oracle's learned-part network (4-layer 3x3x3 conv net on
haloed brick tiles): finite-difference gradients, output definition, loss."""
import numpy as np

import oracle
import synth


def _params(seed, scale=0.2):
    return np.random.default_rng(seed).standard_normal(oracle.net_nparams()) * scale


def test_parameter_count():
    assert oracle.net_nparams() == 27 * 2 * 32 + 32 + 2 * (27 * 32 * 32 + 32) + 27 * 32 * 2 + 2


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    P = _params(2)
    feat = rng.standard_normal((1, 1000, 2))
    tgt = rng.standard_normal((1, 512, 2))
    mask = (rng.uniform(size=(1, 512)) < 0.6).astype(np.uint8)
    loss, g, _ = oracle.net_loss(P, feat, tgt, mask)
    idx = np.concatenate([rng.choice(P.size, 60, replace=False), [0, 1727, 1728, 1759, P.size - 1, P.size - 3]])
    def fd(i, eps):
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += eps
        Pm[i] -= eps
        return (oracle.net_loss(Pp, feat, tgt, mask, grad=False)[0] -
                oracle.net_loss(Pm, feat, tgt, mask, grad=False)[0]) / (2 * eps)

    # central differences at three step sizes: a ReLU kink inside a step
    # spoils that estimate (first-layer weights move many pre-activations, so
    # their kinks are finely spaced), the smallest step avoids it
    for i in idx:
        errs = [abs(fd(i, eps) - g[i]) for eps in (1e-5, 1e-6, 1e-7)]
        assert min(errs) <= 1e-5 * max(1.0, abs(g[i])), (i, errs, g[i])


def test_output_is_a_residual_on_the_tsdf_and_loss_vanishes_at_the_prediction():
    rng = np.random.default_rng(3)
    P = np.zeros(oracle.net_nparams())
    feat = rng.standard_normal((2, 1000, 2))
    tgt = rng.standard_normal((2, 512, 2))
    mask = np.ones((2, 512), np.uint8)
    loss, g, pred = oracle.net_loss(P, feat, tgt, mask)
    # zero weights: mu_hat = tsdf/h at the centre voxel, log s_hat = 0 - log Q_ii
    c = np.array([(lx + 1) + 10 * (ly + 1) + 100 * (lz + 1) for lz in range(8) for ly in range(8) for lx in range(8)])
    np.testing.assert_array_equal(pred[:, :, 0], feat[:, c, 0])
    np.testing.assert_array_equal(pred[:, :, 1], 0.0)
    lq = rng.uniform(0.0, 3.0, (2, 512))
    _, _, pred = oracle.net_loss(P, feat, tgt, mask, lq=lq)
    np.testing.assert_array_equal(pred[:, :, 1], -lq)
    # the baselines shift the outputs only: the gradient is unchanged when the targets shift with them
    P = _params(4)
    _, g0, p0 = oracle.net_loss(P, feat, tgt, mask)
    t1 = tgt.copy()
    t1[:, :, 1] -= lq
    _, g1, p1 = oracle.net_loss(P, feat, t1, mask, lq=lq)
    np.testing.assert_allclose(p1[:, :, 1], p0[:, :, 1] - lq, rtol=0, atol=1e-12)
    np.testing.assert_allclose(g1, g0, rtol=1e-9, atol=1e-12)
    _, _, pred = oracle.net_loss(P, feat, tgt, mask, lq=lq, grad=False)
    loss, g, _ = oracle.net_loss(P, feat, pred, mask, lq=lq)
    assert loss == 0.0 and np.all(g == 0)


def test_features_read_the_band():
    w = synth.make_workload("sphere64", n=24, image_scale=0.5, frames=12)
    b = oracle.build_band_w(w)
    d, hd, _ = oracle.integrate_w(b, w)
    feat = oracle.net_features(b, d)
    assert feat.shape == (b.NB, 1000, 2)
    ijk = b.ijk()
    for v in range(0, b.N, 97):
        r = b.dir[(ijk[v, 0] >> 3) + b.n // 8 * ((ijk[v, 1] >> 3) + b.n // 8 * (ijk[v, 2] >> 3))]
        t = (ijk[v, 0] & 7) + 1 + 10 * ((ijk[v, 1] & 7) + 1) + 100 * ((ijk[v, 2] & 7) + 1)
        assert feat[r, t, 0] == np.float64(b.tsdf[v]) / np.float64(np.float32(b.h))
        assert feat[r, t, 1] == np.log1p(d[v])
    assert np.count_nonzero(feat[:, :, 1]) <= 1000 * b.NB


class _Bricks:
    """Stand-in for a band: the judge reads only NB and the brick offsets."""

    def __init__(self, off):
        self.off = np.asarray(off, np.int64)
        self.NB = len(off) - 1


def test_surrogate_judge_by_hand():
    # brick 0: voxels 0-2, brick 1: voxels 3-6; two probes
    t = np.array([[1.0, 2.0, 3.0, 4.0, 4.0, 1.0, 0.5],
                  [3.0, 2.0, 1.0, 4.0, 4.0, 1.0, 0.5]])
    qd = np.full(7, 1e6)
    s_hat = np.array([2.0, 2.1, 5.0, 4.0, 4.8, 1.0, 0.5])
    stat, acc = oracle.surrogate_judge(_Bricks([0, 3, 7]), np.log(s_hat), t, qd)
    # brick 0: s_J = 2, se = (1, 0, 1), e / f = (0, 0.05, 1.5), e / (3 se + 0.2) = (0, 0.5, 3 / 3.2)
    np.testing.assert_allclose(stat[0], [0.05, 3.0 / 3.2], rtol=1e-12)
    assert acc[0] == 1
    # brick 1: se = 0, e / f = (0, 0.2, 0, 0): median of an even count = mean of the middle two = 0;
    # voxel 4 has e = 0.8 > 3 se + 0.1 f = 0.4
    np.testing.assert_allclose(stat[1], [0.0, 2.0], rtol=1e-12, atol=1e-15)
    assert acc[1] == 0


def test_surrogate_judge_accepts_its_own_mean_and_floors_at_the_diagonal():
    rng = np.random.default_rng(3)
    t = rng.normal(1.0, 0.5, (16, 40))
    qd = np.full(40, 2.0)
    sJ = t.mean(0)
    stat, acc = oracle.surrogate_judge(_Bricks([0, 10, 25, 40]), np.log(np.maximum(sJ, 1e-300)), t, qd)
    pos = sJ > 0
    assert pos.all()
    np.testing.assert_allclose(stat, 0.0, atol=1e-12)
    assert acc.all()
    # a negative probe mean is floored at 1/Q_ii = 0.5: s_hat = 0.5 is then e / f = (0.5 - s_J) / 0.5
    t2 = np.array([[-1.0], [0.6]])
    stat2, _ = oracle.surrogate_judge(_Bricks([0, 1]), np.log([0.5]), t2, np.array([2.0]))
    np.testing.assert_allclose(stat2[0, 0], (0.5 + 0.2) / 0.5, rtol=1e-12)
