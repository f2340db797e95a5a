"""The attention output as the kernels evaluate it, against its definition
(Sec. II-B, DPA-1: O = P V, Y = O Wo + bo with V = G Wv + bv), in FP64 on
the CPU.  With rowsum P = P 1:

  Y = [P G, rowsum P] [Wv Wo; bv Wo] + bo,

and, for dY = dE/dY, the adjoint the kernels run instead of the V form
(dO = dY Wo^T, dV = P^T dO, dP = dO V^T, dE/dG += dV Wv^T):

  dPG = dY [Wv Wo; bv Wo]^T,
  dP = dPG [G 1]^T = dPG[:, :M1] G^T + dPG[:, M1] 1^T,
  dE/dG (through V) = P^T dPG[:, :M1].

The fused 16-bit kernels carry the row-sum column as two ones-columns of the
layer input and the bias product as its 16-bit high and low parts; that
variant is checked too."""

import numpy as np
import pytest


def _case(seed, n=128, nn=87, m1=100, a=128):
    rng = np.random.default_rng(seed)
    P = rng.normal(size=(n, n)) * 0.1
    P[nn:, :] = 0.0  # rows and keys past the last neighbour
    P[:, nn:] = 0.0
    G = rng.normal(size=(n, m1))
    Wv, bv = rng.normal(size=(m1, a)) / np.sqrt(m1), rng.normal(size=a) * 0.1
    Wo, bo = rng.normal(size=(a, m1)) / np.sqrt(a), rng.normal(size=m1) * 0.1
    dY = rng.normal(size=(n, m1))
    return P, G, Wv, bv, Wo, bo, dY


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_forward_identity(seed):
    P, G, Wv, bv, Wo, bo, _ = _case(seed)
    V = G @ Wv + bv
    y_def = (P @ V) @ Wo + bo
    PG1 = np.hstack([P @ G, P.sum(axis=1, keepdims=True)])
    Wvo = np.vstack([Wv @ Wo, bv @ Wo])
    y_pg = PG1 @ Wvo + bo
    assert np.allclose(y_pg, y_def, rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_adjoint_identity(seed):
    P, G, Wv, bv, Wo, bo, dY = _case(seed)
    m1 = G.shape[1]
    # the V form
    V = G @ Wv + bv
    dO = dY @ Wo.T
    dV = P.T @ dO
    dP_def = dO @ V.T
    dG_def = dV @ Wv.T
    # the P G form
    Wvo = np.vstack([Wv @ Wo, bv @ Wo])
    dPG = dY @ Wvo.T  # [n][m1 + 1]
    dP_pg = dPG[:, :m1] @ G.T + dPG[:, m1:m1 + 1]
    dG_pg = P.T @ dPG[:, :m1]
    assert np.allclose(dP_pg, dP_def, rtol=0, atol=1e-11)
    assert np.allclose(dG_pg, dG_def, rtol=0, atol=1e-11)


def test_two_ones_columns_carry_the_bias_product():
    """The fused kernels' form: the layer input has two ones-columns (M1 and
    M1 + 1), so P [G 1 1] has rowsum P twice, and the output weights hold
    bv Wo split into a high part (row M1) and the remainder (row M1 + 1);
    the adjoint's row-sum term is then the sum of the two columns."""
    P, G, Wv, bv, Wo, bo, dY = _case(5)
    m1 = G.shape[1]
    b = bv @ Wo
    b_hi = b.astype(np.float16).astype(np.float64)  # any split with b_hi + b_lo = b
    b_lo = b - b_hi
    G11 = np.hstack([G, np.ones((G.shape[0], 2))])
    Wvo2 = np.vstack([Wv @ Wo, b_hi, b_lo])
    y = (P @ G11) @ Wvo2 + bo
    y_def = (P @ (G @ Wv + bv)) @ Wo + bo
    assert np.allclose(y, y_def, rtol=0, atol=1e-12)
    dPG = dY @ Wvo2.T
    dP = dPG @ G11.T
    dP_def = (dY @ Wo.T) @ (G @ Wv + bv).T
    assert np.allclose(dP, dP_def, rtol=0, atol=1e-11)
    assert np.allclose(P.T @ dPG[:, :m1], (P.T @ (dY @ Wo.T)) @ Wv.T, rtol=0, atol=1e-11)
