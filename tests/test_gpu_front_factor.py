"""The adjoint preconditioner's dense front kernel on its own: the partial LDL^T
of one symmetric front (D and the unit-lower L in the pivot columns, the Schur
complement in the trailing block, and the inverse of L's pivot block) against a
plain FP64 elimination written out here.  Both trailing-update paths are run --
the tensor-core one (TF32 operands split into hi and lo parts, three MMA passes,
FP32 accumulation in TMEM) and the FP32 FMA tiles -- on fronts that span several
128-row tiles with ragged edges, a single pivot column, a partial last panel, on
128/256/512-thread CTAs and with the panel scratch in global memory."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def ldlt_reference(A, p):
    """Right-looking LDL^T of the first p columns, FP64, no pivoting: column k
    keeps d_k on the diagonal and l = a/d_k below; the trailing block loses
    l d_k l^T."""
    W = np.array(A, dtype=np.float64)
    for k in range(p):
        d = W[k, k]
        l = W[k + 1:, k] / d
        W[k + 1:, k + 1:] -= d * np.outer(l, l)
        W[k + 1:, k] = l
    return W


def spd(n, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    return (G @ G.T / n + 0.5 * np.eye(n)).astype(np.float32)


def indefinite(n, seed):
    """Symmetric, diagonally dominant, pivots of both signs."""
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n)) * (0.3 / np.sqrt(n))
    d = rng.uniform(2.0, 3.0, n) * np.where(rng.random(n) < 0.3, -1.0, 1.0)
    return ((B + B.T) / 2 + np.diag(d)).astype(np.float32)


def _errors(A, p, F, Linv):
    W = ldlt_reference(A, p)
    n = A.shape[0]
    low = np.tril(np.ones((n, n), dtype=bool))
    cols = np.zeros((n, n), dtype=bool)
    cols[:, :p] = True
    piv = low & cols
    trail = low & ~cols
    e_piv = np.max(np.abs(F[piv] - W[piv])) / np.max(np.abs(W[piv]))
    e_tr = (np.max(np.abs(F[trail] - W[trail])) / np.max(np.abs(W[trail]))) if trail.any() else 0.0
    L11 = np.tril(W[:p, :p], -1) + np.eye(p)
    X = np.linalg.inv(L11)
    e_inv = np.max(np.abs(np.tril(Linv) - X)) / np.max(np.abs(X))
    upper_zero = np.all(np.triu(Linv, 1) == 0.0)
    return e_piv, e_tr, e_inv, upper_zero


CASES = [  # (n, p, threads, kind)
    (300, 96, 512, "spd"),
    (517, 75, 512, "spd"),
    (640, 200, 512, "indefinite"),
    (200, 200, 256, "spd"),
    (129, 64, 256, "spd"),
    (260, 1, 256, "indefinite"),
    (150, 33, 128, "spd"),
    (384, 130, 256, "indefinite"),
]


@pytest.mark.parametrize("n,p,threads,kind", CASES)
def test_front_factor_against_fp64(n, p, threads, kind):
    from paper_2106_05306_gb300 import front_factor
    A = spd(n, n + p) if kind == "spd" else indefinite(n, n + p)
    res = {}
    for tc in (True, False):
        F, Linv = front_factor(A, p, threads=threads, use_tc=tc)
        e_piv, e_tr, e_inv, uz = _errors(A, p, F, Linv)
        print(f"n {n} p {p} threads {threads} tc {tc}: L/D {e_piv:.2e} Schur {e_tr:.2e} Linv {e_inv:.2e}")
        assert uz
        # FP32 elimination of a well-conditioned front: a few hundred ulps at most
        assert e_piv < 2e-5 and e_tr < 2e-5 and e_inv < 2e-5, (tc, e_piv, e_tr, e_inv)
        res[tc] = F
    # both paths factor the same front; they differ only by rounding
    W = ldlt_reference(A, p)
    low = np.tril(np.ones((n, n), dtype=bool))
    assert np.max(np.abs(res[True][low] - res[False][low])) <= 4e-5 * np.max(np.abs(W[low]))


def test_front_factor_global_scratch_matches_shared():
    """The panel scratch in global memory (fronts too large for shared memory)
    gives the bits of the shared-memory path, on both trailing-update paths."""
    from paper_2106_05306_gb300 import front_factor
    A = spd(700, 7)
    for tc in (True, False):
        F1, X1 = front_factor(A, 160, threads=512, use_tc=tc)
        F2, X2 = front_factor(A, 160, threads=512, use_tc=tc, use_gscr=True)
        assert np.array_equal(F1, F2) and np.array_equal(X1, X2)


def test_front_factor_large_front_global_scratch():
    """A 2000-unknown front (beyond one CTA's shared memory): global scratch."""
    from paper_2106_05306_gb300 import front_factor
    A = spd(2000, 11)
    F, Linv = front_factor(A, 300, threads=512, use_tc=True, use_gscr=True)
    e_piv, e_tr, e_inv, uz = _errors(A, 300, F, Linv)
    print(f"n 2000 p 300 gscr: L/D {e_piv:.2e} Schur {e_tr:.2e} Linv {e_inv:.2e}")
    assert uz and e_piv < 2e-5 and e_tr < 2e-5 and e_inv < 2e-5


def test_front_factor_rejects_bad_sizes():
    from paper_2106_05306_gb300 import front_factor
    from paper_2106_05306_gb300._lib import DCError
    A = spd(64, 1)
    with pytest.raises(DCError):
        front_factor(A, 65)
    with pytest.raises(DCError):
        front_factor(A, 8, threads=96)
