"""The algebra behind the 2D Dirac pulse step (Sec. 2.3, Eqs. 21-26): with a
vector potential in the lattice plane, every merged mixing
M = R(A_P) R(A_{P-1}), R(A) = cos th + i sin th (A/|A|).alpha, keeps the
component pairs (1,4) and (2,3), and its compact form a + i b.alpha + i d.Sigma
has b_3 = d_1 = d_2 = 0, so the real-space pass of the component pairs can apply
it as the 2x2 blocks

    (1,4): [[a + i d3, i (b1 - i b2)], [i (b1 + i b2), a - i d3]]
    (2,3): [[a - i d3, i (b1 + i b2)], [i (b1 - i b2), a + i d3]].

Checked here against 4x4 matrix products built from the Dirac matrices, with
a, b, d read off by traces (tr(alpha_j alpha_k) = 4 delta_jk, tr(alpha_j) =
tr(Sigma_k alpha_j) = 0).  No GPU, no library code."""
import numpy as np
import pytest

S1 = np.array([[0, 1], [1, 0]], dtype=complex)
S2 = np.array([[0, -1j], [1j, 0]], dtype=complex)
S3 = np.array([[1, 0], [0, -1]], dtype=complex)
Z = np.zeros((2, 2), dtype=complex)
ALPHA = [np.block([[Z, s], [s, Z]]) for s in (S1, S2, S3)]   # Dirac representation
SIGMA = [np.block([[s, Z], [Z, s]]) for s in (S1, S2, S3)]


def R(A, c=137.036, q=-1.0, tau=1e-3, hbar=1.0):
    """Half-step mixing exp(i th (A/|A|).alpha) with th = q c |A| tau / (2 hbar)."""
    A = np.asarray(A, dtype=float)
    mag = np.linalg.norm(A)
    th = 0.5 * q * c * mag * tau / hbar
    M = np.cos(th) * np.eye(4, dtype=complex)
    if mag > 0:
        M = M + 1j * np.sin(th) * sum(A[k] / mag * ALPHA[k] for k in range(3))
    return M


def compact(M):
    """(a, b, d) with M = a + i b.alpha + i d.Sigma (a, b, d real for these M)."""
    a = np.trace(M) / 4
    b = [np.trace(ALPHA[k] @ M) / 4j for k in range(3)]
    d = [np.trace(SIGMA[k] @ M) / 4j for k in range(3)]
    return a, np.array(b), np.array(d)


@pytest.mark.parametrize("seed", range(6))
def test_in_plane_mixing_keeps_the_pairs_and_matches_the_blocks(seed):
    rng = np.random.default_rng(seed)
    Ap = np.array([*rng.normal(0, 30, 2), 0.0])
    Aq = np.array([*rng.normal(0, 30, 2), 0.0])
    M = R(Ap) @ R(Aq)
    a, b, d = compact(M)
    # the compact form reproduces M and is real
    rebuilt = a * np.eye(4) + 1j * sum(b[k] * ALPHA[k] for k in range(3)) + 1j * sum(d[k] * SIGMA[k] for k in range(3))
    assert np.abs(rebuilt - M).max() < 1e-13
    assert abs(a.imag) < 1e-14 and np.abs(b.imag).max() < 1e-14 and np.abs(d.imag).max() < 1e-14
    a, b, d = a.real, b.real, d.real
    # in-plane A: no alpha_3 part, Sigma only along e_3 (d = A_P x A_{P-1} direction)
    assert abs(b[2]) < 1e-14 and abs(d[0]) < 1e-14 and abs(d[1]) < 1e-14
    assert abs(d[2]) > 1e-6   # non-parallel fields: the Sigma_3 term is present
    # the pairs (1,4) and (2,3) (indices 0,3 and 1,2) do not mix
    for i in (0, 3):
        for j in (1, 2):
            assert abs(M[i, j]) < 1e-14 and abs(M[j, i]) < 1e-14
    b1, b2, d3 = b[0], b[1], d[2]
    blk14 = np.array([[a + 1j * d3, 1j * (b1 - 1j * b2)], [1j * (b1 + 1j * b2), a - 1j * d3]])
    blk23 = np.array([[a - 1j * d3, 1j * (b1 + 1j * b2)], [1j * (b1 - 1j * b2), a + 1j * d3]])
    assert np.abs(M[np.ix_([0, 3], [0, 3])] - blk14).max() < 1e-13
    assert np.abs(M[np.ix_([1, 2], [1, 2])] - blk23).max() < 1e-13


def test_out_of_plane_field_breaks_the_pairs():
    """A_3 != 0 couples the pairs (so the pair pass must not take such rows)."""
    M = R([10.0, -4.0, 7.0]) @ R([3.0, 8.0, -2.0])
    a, b, d = compact(M)
    assert abs(b[2]) > 1e-6 or abs(d[0]) > 1e-6 or abs(d[1]) > 1e-6
    assert abs(M[0, 2]) > 1e-9 or abs(M[0, 1]) > 1e-9
