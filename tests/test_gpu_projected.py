"""The Davidson solvers' projected eigensolver (the Rayleigh-Ritz step of Sec. 2.2
Step 3 on the search space) through hinqs_selftest_projected_eig, on pencils whose
eigenpairs LAPACK gives: the lowest pair to FP64 accuracy on every path (no S, S near
the identity, general S; FP32 Jacobi refined in FP64, FP64 Jacobi for a (near-)
degenerate lowest pair), the other pairs to the FP32 solve's accuracy."""
import numpy as np
import pytest
import scipy.linalg

hq = pytest.importorskip("paper_2606_26760_b300")
pytestmark = pytest.mark.gpu

SERIES, CHOLESKY, REFINED = 1, 2, 4


def pencil(m, seed, gap=None, s_kind=None):
    """A pencil (G, S) whose eigenvalues are spread over [-30, 10] (a chosen gap between
    the lowest two), with S None, near the identity (an FP32-orthonormal basis) or a
    general SPD matrix: G = R A R^T for S = R R^T and A with those eigenvalues."""
    rng = np.random.default_rng(seed)
    w = np.sort(rng.uniform(-30.0, 10.0, m))
    if gap is not None and m > 1:
        w[1] = w[0] + gap
        w = np.sort(w)
    Q, _ = np.linalg.qr(rng.normal(size=(m, m)))
    A = Q @ np.diag(w) @ Q.T
    if s_kind is None:
        S = None
    elif s_kind == "near":
        E = rng.uniform(-1e-7, 1e-7, (m, m))
        S = np.eye(m) + 0.5 * (E + E.T)
    else:
        B = rng.normal(size=(m, m))
        S = B @ B.T / m + 0.5 * np.eye(m)
    R = np.eye(m) if S is None else np.linalg.cholesky(S)
    G = R @ A @ R.T
    return 0.5 * (G + G.T), S


def check_lowest(G, S, theta, y):
    Sm = np.eye(len(G)) if S is None else S
    lam = scipy.linalg.eigh(G, Sm, eigvals_only=True)
    scale = np.max(np.abs(lam))
    assert abs(theta - lam[0]) <= 1e-12 * scale
    assert abs(y @ Sm @ y - 1.0) <= 1e-12
    assert np.linalg.norm(G @ y - theta * (Sm @ y)) <= 1e-11 * scale
    big = np.argmax(np.abs(y))
    assert y[big] > 0
    return lam


@pytest.mark.parametrize("m", [1, 2, 7, 16, 32])
def test_no_overlap_matrix(m):
    G, S = pencil(m, 10 + m)
    theta, y, _, path = hq.selftest_projected_eig(G)
    check_lowest(G, S, theta, y)
    assert path == REFINED


@pytest.mark.parametrize("m", [1, 5, 12, 32])
def test_overlap_near_identity_takes_the_series(m):
    G, S = pencil(m, 20 + m, s_kind="near")
    theta, y, _, path = hq.selftest_projected_eig(G, S)
    check_lowest(G, S, theta, y)
    assert path == SERIES | REFINED


@pytest.mark.parametrize("m", [1, 6, 17])
def test_general_overlap_takes_cholesky(m):
    G, S = pencil(m, 30 + m, s_kind="spd")
    theta, y, _, path = hq.selftest_projected_eig(G, S)
    check_lowest(G, S, theta, y)
    assert path == CHOLESKY | REFINED


@pytest.mark.parametrize("gap,s_kind", [(0.0, None), (1e-9, None), (0.0, "near"), (1e-8, "spd")])
def test_degenerate_lowest_pair_takes_fp64_jacobi(gap, s_kind):
    """Two lowest eigenvalues closer than FP32 resolves: the FP64 Jacobi path, and the
    pair still to FP64 accuracy (y any vector of the two-dimensional eigenspace)."""
    G, S = pencil(9, 40, gap=gap, s_kind=s_kind)
    theta, y, _, path = hq.selftest_projected_eig(G, S)
    check_lowest(G, S, theta, y)
    assert not path & REFINED


@pytest.mark.parametrize("s_kind", [None, "near", "spd"])
def test_every_pair_ascending(s_kind):
    m = 14
    G, S = pencil(m, 50, s_kind=s_kind)
    Sm = np.eye(m) if S is None else S
    theta, y, pairs, _ = hq.selftest_projected_eig(G, S, want_pairs=True)
    lam = scipy.linalg.eigh(G, Sm, eigvals_only=True)
    scale = np.max(np.abs(lam))
    assert np.all(np.diff(pairs[:, 0]) >= 0)
    assert np.max(np.abs(pairs[:, 0] - lam)) <= 1e-5 * scale
    assert pairs[0, 0] == theta and np.allclose(np.abs(pairs[0, 1:]), np.abs(y), rtol=0, atol=1e-15)
    for j in range(m):
        v = pairs[j, 1:]
        assert abs(v @ Sm @ v - 1.0) <= 1e-5
        assert np.linalg.norm(G @ v - pairs[j, 0] * (Sm @ v)) <= 1e-4 * scale


def test_argument_errors():
    G = np.eye(3)
    with pytest.raises(RuntimeError):
        hq.selftest_projected_eig(np.eye(33))
    with pytest.raises(RuntimeError):
        hq.selftest_projected_eig(np.zeros((0, 0)))
    theta, y, _, _ = hq.selftest_projected_eig(G)
    assert theta == 1.0
