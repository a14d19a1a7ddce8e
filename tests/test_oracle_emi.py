"""Pins for the oracle's coherence, EMI phase linking, gamma_t and compression.

Closed forms (N=2, consistent-phase coherence, rank one), invariants
(Hermitian, unit diagonal, PSD; equivariance under per-date phase screens and
scalings), brute force on tiny windows, and a library eigensolver on the
matrix the paper's eq. (emi-eigenvalue-problem) names.
"""
import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(1234)


def wrapped(a):
    return np.angle(np.exp(1j * a))


def full_from_packed(Cp, N):
    M = np.zeros((N, N), complex)
    idx = 0
    for i in range(N):
        for k in range(i, N):
            M[i, k] = Cp[idx]
            M[k, i] = np.conj(Cp[idx])
            idx += 1
    return M


def packed_from_full(M):
    N = M.shape[0]
    return np.array([M[i, k] for i in range(N) for k in range(i, N)])


def rand_stack(N, H, W, rng=RNG):
    return (rng.standard_normal((N, H, W)) + 1j * rng.standard_normal((N, H, W))) / np.sqrt(2)


def all_ones_mask(H, W, window):
    wy, wx, sy, sx = window
    P = np.ones((H, W), np.float32)
    return oracle.shp_select(P, window, np.float32(2.0))[0]


# --------------------------------------------------------------- coherence

def test_covariance_brute_force_tiny():
    N, H, W = 3, 6, 8
    window = (3, 5, 2, 3)
    z = rand_stack(N, H, W)
    rng = np.random.default_rng(5)
    P = rng.gamma(4.0, 1.0, size=(H, W)).astype(np.float32)
    mask, count = oracle.shp_select(P, window, np.float32(2.5))
    C = oracle.covariance(z, window, mask)
    Ho, Wo = H // 2, W // 3
    for i in range(Ho):
        for j in range(Wo):
            cy, cx = i * 2 + 1, j * 3 + 1
            S = np.zeros((N, N), complex)
            L = 0
            for dy in range(-1, 2):
                for dx in range(-2, 3):
                    b = (dy + 1) * 5 + dx + 2
                    if (int(mask[i, j, 0]) >> b) & 1:
                        v = z[:, cy + dy, cx + dx]
                        S += np.outer(v, v.conj())
                        L += 1
            assert L == count[i, j]
            d = np.sqrt(np.real(np.diag(S)))
            want = S / np.outer(d, d)
            np.fill_diagonal(want, 1.0)
            np.testing.assert_allclose(full_from_packed(C[i, j], N), want, rtol=1e-12, atol=1e-14)


def test_covariance_hermitian_psd_unit_diagonal():
    N, H, W = 8, 20, 30
    window = (5, 11, 1, 1)
    z = rand_stack(N, H, W)
    C = oracle.covariance(z, window, all_ones_mask(H, W, window))
    for i in range(0, H, 3):
        for j in range(0, W, 4):
            M = full_from_packed(C[i, j], N)
            assert np.allclose(np.diag(M), 1.0, atol=0)
            assert np.all(np.abs(M) <= 1.0 + 1e-12)
            assert np.linalg.eigvalsh(M).min() >= -1e-12


def test_covariance_fully_coherent_closed_form():
    N, H, W = 6, 10, 12
    phi = RNG.uniform(-np.pi, np.pi, N)
    amp = RNG.rayleigh(1.0, (H, W)) + 0.1
    z = amp[None] * np.exp(1j * phi)[:, None, None] * np.exp(1j * RNG.uniform(-3, 3, (H, W)))[None]
    window = (3, 5, 1, 1)
    C = oracle.covariance(z, window, all_ones_mask(H, W, window))
    want = np.exp(1j * (phi[:, None] - phi[None, :]))
    for i in range(H):
        for j in range(W):
            np.testing.assert_allclose(full_from_packed(C[i, j], N), want, atol=1e-12)


def test_covariance_scale_and_phase_screen_equivariance():
    N, H, W = 5, 9, 15
    window = (3, 5, 1, 1)
    z = rand_stack(N, H, W)
    m = all_ones_mask(H, W, window)
    C0 = oracle.covariance(z, window, m)
    s = RNG.uniform(0.2, 5.0, N)
    beta = RNG.uniform(-np.pi, np.pi, N)
    C1 = oracle.covariance(z * (s * np.exp(1j * beta))[:, None, None], window, m)
    rot = packed_from_full(np.exp(1j * (beta[:, None] - beta[None, :])))
    np.testing.assert_allclose(C1, C0 * rot[None, None], atol=1e-12)


def test_covariance_no_data_is_nan():
    N, H, W = 3, 5, 5
    z = rand_stack(N, H, W)
    P = np.ones((H, W), np.float32)
    P[2, 2] = 0
    mask, count = oracle.shp_select(P, (3, 3, 1, 1), np.float32(2.0))
    C = oracle.covariance(z, (3, 3, 1, 1), mask)
    assert np.all(np.isnan(C[2, 2]))
    assert not np.any(np.isnan(C[0, 0]))


# --------------------------------------------------------------------- EMI

def test_emi_n2_closed_form():
    # For N=2, |C|^-1 o C has eigenvalues (1 +- g^2)/(1 - g^2); the smallest is
    # 1, with eigenvector (1, e^{-j theta}) for C_01 = g e^{j theta}: the linked
    # phase equals the interferogram phase, and gamma_t = 1 (Sec. III-C).
    gs = RNG.uniform(0.05, 0.95, 200)
    th = RNG.uniform(-np.pi, np.pi, 200)
    C = np.stack([np.ones(200), gs * np.exp(1j * th), np.ones(200)], axis=1)
    out = oracle.phase_link(C, 2, ref=0)
    assert np.all(out["status"] == 0)
    np.testing.assert_allclose(out["phase"][0], 0.0, atol=0)
    np.testing.assert_allclose(wrapped(out["phase"][1] - np.angle(np.conj(C[:, 1]))), 0, atol=1e-12)
    np.testing.assert_allclose(out["lam"], 1.0, atol=1e-12)
    np.testing.assert_allclose(out["tcoh"], 1.0, atol=1e-12)
    out1 = oracle.phase_link(C, 2, ref=1)
    np.testing.assert_allclose(out1["phase"][1], 0.0, atol=0)
    np.testing.assert_allclose(wrapped(out1["phase"][0] - np.angle(C[:, 1])), 0, atol=1e-12)


def exp_coherence(N, tau, rinf=0.1, rho0=0.7):
    t = 12.0 * np.arange(N)
    R = rinf + (rho0 - rinf) * np.exp(-np.abs(t[:, None] - t[None]) / tau)
    np.fill_diagonal(R, 1.0)
    return R


@pytest.mark.parametrize("N", [3, 5, 10, 15, 21, 30])
def test_emi_consistent_phase_recovers_truth(N):
    # C = Phi R Phi^H with R real, positive, PD and unit diagonal: |C| = R and
    # |C|^-1 o C = Phi (R^-1 o R) Phi^H, whose smallest eigenvalue is 1 with
    # eigenvector Phi 1 (Fiedler: R^-1 o R - I is PSD; its row sums are 1).
    R = exp_coherence(N, RNG.uniform(12, 120))
    phi = RNG.uniform(-np.pi, np.pi, N)
    C = np.exp(1j * (phi[:, None] - phi[None])) * R
    for ref in (0, N // 2, N - 1):
        out = oracle.phase_link(packed_from_full(C)[None], N, ref=ref)
        assert out["status"][0] == 0
        np.testing.assert_allclose(wrapped(out["phase"][:, 0] - (phi - phi[ref])), 0, atol=1e-9)
        assert out["phase"][ref, 0] == 0.0
        assert out["lam"][0] == pytest.approx(1.0, abs=1e-10)
        assert out["tcoh"][0] == pytest.approx(1.0, abs=1e-12)


def test_emi_matches_library_eigensolver_on_random_coherence():
    N, H, W = 7, 12, 16
    window = (5, 11, 1, 1)
    z = rand_stack(N, H, W)
    C = oracle.covariance(z, window, all_ones_mask(H, W, window)).reshape(-1, N * (N + 1) // 2)
    out = oracle.phase_link(C, N, ref=2, cond=True)
    for p in range(C.shape[0]):
        M = full_from_packed(C[p], N)
        G = np.abs(M)
        A = np.linalg.inv(G) * M
        w, V = np.linalg.eigh(A)
        v = V[:, 0]
        want = np.angle(v * np.conj(v[2]))
        assert out["status"][p] == 0
        np.testing.assert_allclose(out["lam"][p], w[0], rtol=1e-10)
        np.testing.assert_allclose(out["gap"][p], w[1] - w[0], rtol=1e-8, atol=1e-12)
        np.testing.assert_allclose(wrapped(out["phase"][:, p] - want), 0, atol=1e-8)
        ge = np.linalg.eigvalsh(G)
        np.testing.assert_allclose(out["condG"][p], ge[-1] / ge[0], rtol=1e-8)


@pytest.mark.parametrize("beta", [0.1, 0.5, 0.9])
def test_regularised_emi_matches_library_eigensolver(beta):
    # Sec. III-B's regularisation G = (1 - beta)|C| + beta I: the smallest
    # eigenvector of G^-1 o C written out with numpy's inverse and eigh.
    N, H, W = 7, 12, 16
    window = (5, 11, 1, 1)
    z = rand_stack(N, H, W, np.random.default_rng(3))
    C = oracle.covariance(z, window, all_ones_mask(H, W, window)).reshape(-1, N * (N + 1) // 2)
    out = oracle.phase_link(C, N, ref=2, beta=beta)
    for p in range(C.shape[0]):
        M = full_from_packed(C[p], N)
        G = (1 - beta) * np.abs(M) + beta * np.eye(N)
        w, V = np.linalg.eigh(np.linalg.inv(G) * M)
        v = V[:, 0]
        assert out["status"][p] == 0
        np.testing.assert_allclose(out["lam"][p], w[0], rtol=1e-10)
        np.testing.assert_allclose(wrapped(out["phase"][:, p] - np.angle(v * np.conj(v[2]))), 0, atol=1e-9)


def test_regularisation_limit_beta_to_one():
    # G^-1 = (1/beta)(I - ((1 - beta)/beta)|C|_off) + O((1 - beta)^2), so as
    # beta -> 1 the smallest eigenvector of G^-1 o C tends to the largest one of
    # |C| o C with its diagonal removed, the phase error shrinking like 1 - beta.
    N, H, W = 7, 12, 16
    window = (5, 11, 1, 1)
    z = rand_stack(N, H, W, np.random.default_rng(3))
    C = oracle.covariance(z, window, all_ones_mask(H, W, window)).reshape(-1, N * (N + 1) // 2)
    errs = {}
    for beta in (0.999, 0.9999):
        out = oracle.phase_link(C, N, ref=2, beta=beta)
        e = []
        for p in range(C.shape[0]):
            M = full_from_packed(C[p], N)
            K = np.abs(M) * M
            np.fill_diagonal(K, 0)
            v = np.linalg.eigh(K)[1][:, -1]
            e.append(np.abs(wrapped(out["phase"][:, p] - np.angle(v * np.conj(v[2])))).max())
        errs[beta] = max(e)
    assert errs[0.9999] < 1e-3
    assert 5 < errs[0.999] / errs[0.9999] < 20


def test_emi_rank_one_falls_back_to_evd():
    # One look: C = z z^H / |z_i||z_k|, |C| is the all-ones matrix (singular):
    # the inversion fails and the EVD fallback returns the phases of z.
    N = 9
    z = RNG.standard_normal(N) + 1j * RNG.standard_normal(N)
    u = z / np.abs(z)
    C = np.outer(u, u.conj())
    out = oracle.phase_link(packed_from_full(C)[None], N, ref=0)
    assert out["status"][0] == 2
    assert np.isnan(out["lam"][0])
    np.testing.assert_allclose(wrapped(out["phase"][:, 0] - np.angle(z * np.conj(z[0]))), 0, atol=1e-10)
    assert out["tcoh"][0] == pytest.approx(1.0, abs=1e-12)


def test_evd_fallback_matches_library_eigensolver():
    # A rank-deficient C with |C| singular: two identical dates.
    N = 6
    rng = np.random.default_rng(7)
    Z = rng.standard_normal((N, 40)) + 1j * rng.standard_normal((N, 40))
    Z[3] = Z[1] * np.exp(0.7j)
    S = Z @ Z.conj().T
    d = np.sqrt(np.real(np.diag(S)))
    C = S / np.outer(d, d)
    np.fill_diagonal(C, 1.0)
    out = oracle.phase_link(packed_from_full(C)[None], N, ref=0)
    assert out["status"][0] == 2
    w, V = np.linalg.eigh(C)
    v = V[:, -1]
    np.testing.assert_allclose(wrapped(out["phase"][:, 0] - np.angle(v * np.conj(v[0]))), 0, atol=1e-9)


def test_emi_equivariant_under_phase_screen():
    N, H, W = 6, 10, 14
    window = (3, 5, 1, 1)
    z = rand_stack(N, H, W)
    m = all_ones_mask(H, W, window)
    beta = RNG.uniform(-np.pi, np.pi, N)
    C0 = oracle.covariance(z, window, m).reshape(-1, 21)
    C1 = oracle.covariance(z * np.exp(1j * beta)[:, None, None], window, m).reshape(-1, 21)
    o0 = oracle.phase_link(C0, N, ref=1)
    o1 = oracle.phase_link(C1, N, ref=1)
    d = wrapped(o1["phase"] - o0["phase"] - (beta - beta[1])[:, None])
    np.testing.assert_allclose(d, 0, atol=1e-9)
    np.testing.assert_allclose(o1["tcoh"], o0["tcoh"], atol=1e-12)


def test_no_data_phase_link():
    C = np.full((1, 6), np.nan + 0j)
    out = oracle.phase_link(C, 3, ref=0)
    assert out["status"][0] == 3 and np.all(np.isnan(out["phase"]))


# ------------------------------------------------------------------- gamma_t

def test_temporal_coherence_closed_forms():
    # N=2: a single interferogram always fits exactly (Sec. III-C).
    C = np.array([1.0, 0.3 * np.exp(0.4j), 1.0])
    for ph in ([0.0, 1.0], [0.2, -2.0]):
        assert oracle.temporal_coherence(C, np.array(ph)) == pytest.approx(1.0, abs=1e-15)
    # N=3 with linked phases all zero: |e^{ja} + e^{jb} + e^{jc}| / 3.
    a, b, c = 0.3, -1.1, 2.0
    Cp = np.array([1, 0.5 * np.exp(1j * a), 0.4 * np.exp(1j * b), 1, 0.9 * np.exp(1j * c), 1])
    want = abs(np.exp(1j * a) + np.exp(1j * b) + np.exp(1j * c)) / 3
    assert oracle.temporal_coherence(Cp, np.zeros(3)) == pytest.approx(want, abs=1e-15)
    # phihat_ik = phihat_i - phihat_k enters with a minus sign.
    ph = np.array([0.0, 0.3, -0.2])
    want = abs(np.exp(1j * (a - (ph[0] - ph[1]))) + np.exp(1j * (b - (ph[0] - ph[2])))
               + np.exp(1j * (c - (ph[1] - ph[2])))) / 3
    assert oracle.temporal_coherence(Cp, ph) == pytest.approx(want, abs=1e-15)
    # An exactly-zero entry contributes exp(-j phihat_ik).
    Cz = np.array([1, 0.0, 1.0])
    assert oracle.temporal_coherence(Cz, np.array([0.0, 0.5])) == pytest.approx(1.0, abs=1e-15)


# ----------------------------------------------------------------- compress

def test_compress_noise_free_closed_form():
    # z_i = a e^{j phi_i} and phihat = phi - phi_r: kappa = M a e^{j phi_r}
    # (the base phase of Sec. II-B).
    N, H, W = 5, 7, 9
    phi = RNG.uniform(-np.pi, np.pi, N)
    a = RNG.rayleigh(1.0, (H, W))
    z = a[None] * np.exp(1j * phi)[:, None, None]
    r = 0
    ph = np.broadcast_to((phi - phi[r])[:, None, None], (N, H, W)).copy()
    k = oracle.compress(z, 0, (1, 1, 1, 1), ph)
    np.testing.assert_allclose(k, N * a * np.exp(1j * phi[r]), rtol=1e-12)


def test_compress_common_rotation_and_cells():
    N, H, W, sy, sx = 3, 11, 20, 3, 6
    Ho, Wo = H // sy, W // sx
    z = rand_stack(N, H, W)
    ph = RNG.uniform(-np.pi, np.pi, (N, Ho, Wo))
    k0 = oracle.compress(z, 1, (3, 5, sy, sx), ph)
    k1 = oracle.compress(z, 1, (3, 5, sy, sx), ph + 0.8)
    np.testing.assert_allclose(k1, k0 * np.exp(-0.8j), atol=1e-12)
    for y in range(H):
        for x in range(W):
            ci, cj = min(y // sy, Ho - 1), min(x // sx, Wo - 1)
            want = sum(np.exp(-1j * ph[i, ci, cj]) * z[i, y, x] for i in (1, 2))
            assert abs(k0[y, x] - want) < 1e-12


def test_compress_no_data_cell_is_zero():
    z = rand_stack(2, 4, 4)
    ph = np.zeros((2, 4, 4))
    ph[:, 1, 2] = np.nan
    k = oracle.compress(z, 0, (1, 1, 1, 1), ph)
    assert k[1, 2] == 0 and np.all(k[0] != 0)


def test_inversion_failure_threshold():
    # Sec. III-B's "inversion fails due to numerical issues", read as a Cholesky
    # pivot of the unit-diagonal |C| at or below 1e-4: for N=2 the second pivot is
    # exactly 1 - g^2.  Both answers have the interferogram phase for N=2; the
    # status tells which branch ran.
    for pivot, want in ((2e-4, 0), (1.5e-4, 0), (5e-5, 2), (0.0, 2)):
        g = np.sqrt(1.0 - pivot)
        C = np.array([[1.0, g * np.exp(0.3j), 1.0]])
        out = oracle.phase_link(C, 2, ref=0)
        assert out["status"][0] == want, (pivot, out["status"][0])
        assert abs(wrapped(out["phase"][1, 0] + 0.3)) < 1e-9
