"""The FP64-class complex products behind the refinement residuals, called directly
(fosb_zgemm_fp64class) on the operands of the exact-arithmetic method check: rows and
columns spread over 10^+-3 with a dominant diagonal, compared with the exact rational product
per entry relative to sum |Z||X|, at each method's bound: 4e-15 for the digit splitting (the
truncation of seven digits, independent of K), K 2^-48 for float-float (48-bit operands and
one rounding of that size per accumulation step); on the method check's 12 x 6 x 64 case and
on ragged sizes that leave partial tiles in every dimension."""
import math
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_01457_gb300 as mod

    mod.build.build()
    return mod


def _operands(M, N, K, seed=3):
    rng = np.random.default_rng(seed)
    rs = 10.0 ** rng.uniform(-3, 3, M)
    cs = 10.0 ** rng.uniform(-3, 3, N)
    Z = (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))) * rs[:, None]
    for i in range(min(M, K)):
        Z[i, i] = complex(50 * Z[i, i].real, Z[i, i].imag)
    X = (rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))) * cs[None, :]
    return Z, X


def _worst(Z, X, C):
    M, K = Z.shape
    N = X.shape[1]
    worst = 0.0
    for i in range(M):
        for j in range(N):
            er = sum(Fraction(Z[i, k].real) * Fraction(X[k, j].real) - Fraction(Z[i, k].imag) * Fraction(X[k, j].imag)
                     for k in range(K))
            ei = sum(Fraction(Z[i, k].real) * Fraction(X[k, j].imag) + Fraction(Z[i, k].imag) * Fraction(X[k, j].real)
                     for k in range(K))
            err = math.hypot(float(Fraction(C[i, j].real) - er), float(Fraction(C[i, j].imag) - ei))
            worst = max(worst, err / float(np.sum(np.abs(Z[i]) * np.abs(X[:, j]))))
    return worst


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("shape", [(12, 6, 64), (37, 11, 150)])
def test_fp64_class_product_against_exact_rational_product(F, method, shape):
    M, N, K = shape
    Z, X = _operands(M, N, K)
    Zd = torch.tensor(Z, dtype=torch.complex128, device="cuda")
    Xd = torch.tensor(X, dtype=torch.complex128, device="cuda")
    Cd = torch.full((M, N), 3.0, dtype=torch.complex128, device="cuda")  # overwritten
    F.zgemm_fp64class(Zd, Xd, Cd, method=method)
    bound = 4e-15 if method == 0 else K * 2.0**-48
    assert _worst(Z, X, Cd.cpu().numpy()) < bound
