"""FP64 measurement probes through the C ABI: both squaring routines (the
forward kernels' DFMA routine and the DMMA tile routine) compute the restored
squarings of the propagator's symmetric form, checked against plain numpy on
the same matrices; the throughput probe runs and counts its FLOPs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dx():
    import torch  # noqa: F401
    from paper_2509_25347_gb300 import build
    build.build()
    import paper_2509_25347_gb300 as m
    m.load_library()
    m.get_status()
    return m


def symmetric_propagators(n, nmat, seed):
    """E = exp(2^-s S) for random symmetric arrowheads S = D_sigma A D_sigma^-1
    (A = dt Omega_v of Eq. jacobian), with their sigma: E sigma = sigma."""
    rng = np.random.default_rng(seed)
    E = np.empty((nmat, n, n))
    sig = np.empty((nmat, n))
    for m in range(nmat):
        eps = 10.0 ** rng.uniform(-2, 0, n - 1)
        alpha = 10.0 ** rng.uniform(-1, 1, n - 1)
        S = np.zeros((n, n))
        S[0, 0] = -np.sum(eps * alpha)
        S[0, 1:] = S[1:, 0] = np.sqrt(eps) * alpha
        S[1:, 1:] = np.diag(-alpha)
        lam, Q = np.linalg.eigh(S / 2.0 ** 6)
        E[m] = (Q * np.exp(lam)) @ Q.T
        sig[m] = np.concatenate([[1.0], np.sqrt(eps)])
    return E, sig


def restored_squarings(E, sig, reps):
    E = E.copy()
    for _ in range(reps):
        E = E @ E
        for i in range(E.shape[0]):
            off = np.delete(E[i], i) @ np.delete(sig, i)
            E[i, i] = 1.0 - off / sig[i]
    return E


@pytest.mark.parametrize("n", [2, 5, 9, 17, 24])
def test_probe_square_both_kinds_match_numpy(dx, n):
    import torch
    E, sig = symmetric_propagators(n, 37, seed=n)
    reps = 4
    ref = np.stack([restored_squarings(E[m], sig[m], reps) for m in range(E.shape[0])])
    tE, ts = torch.from_numpy(E).cuda(), torch.from_numpy(sig).cuda()
    for kind in ("dfma", "dmma"):
        got = dx.probe_square(tE, ts, reps, kind=kind).cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref)), kind
        assert np.allclose(got, np.transpose(got, (0, 2, 1)), rtol=0, atol=1e-15), kind


def test_probe_fp64_rate_runs(dx):
    import torch
    for kind in ("dfma", "dmma"):
        flop = dx.probe_fp64_rate(kind, iters=64)
        torch.cuda.synchronize()
        assert flop > 0
    assert dx.get_status() == 0
