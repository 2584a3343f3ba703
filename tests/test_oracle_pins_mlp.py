"""Pin of the numpy reference of the guess network: its analytic gradient against
central finite differences in FP64 (the paper has no network; this pins the oracle to
the definition of the loss, not to itself)."""
import numpy as np

from oracle import mlp_oracle as M


def test_mlp_oracle_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    F, H, O, n = 5, 7, 3, 11
    npar = H * F + H + 2 * (H * H + H) + O * H + O
    p = rng.normal(0, 0.5, npar)
    norm = np.concatenate([rng.normal(0, 1, F), rng.uniform(0.5, 2, F), rng.normal(0, 1, O), rng.uniform(0.5, 2, O)])
    X = rng.normal(0, 1, (n, F))
    Y = rng.normal(0, 1, (n, O))
    loss, g = M.loss_grad(p, norm, X, Y, F, H, O)
    h = 1e-6
    for k in rng.choice(npar, 40, replace=False):
        e = np.zeros(npar)
        e[k] = h
        fd = (M.loss_grad(p + e, norm, X, Y, F, H, O)[0] - M.loss_grad(p - e, norm, X, Y, F, H, O)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(fd)), (k, fd, g[k])
    # the loss is the mean squared error of the normalised outputs
    y_hat = (M.predict(p, norm, X, F, H, O) - norm[2 * F:2 * F + O]) / norm[2 * F + O:]
    t = (Y - norm[2 * F:2 * F + O]) / norm[2 * F + O:]
    assert abs(loss - ((y_hat - t) ** 2).mean()) < 1e-14
