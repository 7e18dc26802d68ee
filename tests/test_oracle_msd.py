"""Pins of the multi-determinant trial oracle (oracle/msd.py; Sec. V: |psi_T> = sum_I c_I |D_I>,
orthogonal CI or non-orthogonal with <D_I|D_J> = S_IJ).

* Overlap, local energy, force-bias traces and the energy shift E_T (the place where S_IJ
  enters; the variational energy of a non-orthogonal expansion) against brute-force Fock-space
  vectors sum_I c_I |D_I>.
* One determinant and a repeated determinant reduce to the single-determinant functions; a
  re-gauged expansion (D_I -> D_I R_I, c_I -> c_I / det R_I: the same state) changes nothing.
* The phaseless step runs with the expansion, and a one-determinant expansion reproduces the
  single-determinant trajectory."""
import numpy as np

from oracle import afqmc as O
from oracle.fock import FockSpace, four_index_from_cholesky
from oracle.msd import MSDTrial, determinant_matrix_elements
from paper_2003_01831_gb300 import synthetic as syn


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def system(seed, M=5, Nup=2, Ndn=2, nch=4, ND=3):
    rng = np.random.default_rng(seed)
    h, L, _ = syn.make_hamiltonian(M, nch, rng)
    ham = O.Hamiltonian(h=h, L=L, E0=0.4)
    dets = [(crandn(rng, M, Nup), crandn(rng, M, Ndn)) for _ in range(ND)]
    c = crandn(rng, ND)
    Phi = [crandn(rng, 3, M, Nup), crandn(rng, 3, M, Ndn)]
    return ham, MSDTrial(dets, c), Phi, rng


def fock_vector(fs, trial):
    return sum(c * fs.slater_vector(*D) for c, D in zip(trial.c, trial.dets))


def test_mixed_estimates_against_fock_space():
    ham, trial, Phi, _ = system(3)
    fs = FockSpace(5, 2, 2)
    H = fs.hamiltonian(ham.h, four_index_from_cholesky(ham.L), ham.E0)
    vp = fock_vector(fs, trial)
    lo = trial.log_overlap(Phi)
    E, t = trial.local_energy(ham, Phi)
    for w in range(3):
        vf = fs.slater_vector(Phi[0][w], Phi[1][w])
        ov = np.vdot(vp, vf)
        assert abs(np.exp(lo[w]) - ov) < 1e-12 * abs(ov)
        ref = np.vdot(vp, H @ vf) / ov
        assert abs(E[w] - ref) < 1e-11 * max(1.0, abs(ref)), w
        for n in range(ham.Nchol):
            tref = np.vdot(vp, fs.one_body_operator(ham.L[n]) @ vf) / ov
            assert abs(t[w, n] - tref) < 1e-11 * max(1.0, abs(tref)), (w, n)
    Ev = np.vdot(vp, H @ vp) / np.vdot(vp, vp)
    assert abs(trial.energy_shift(ham) - Ev) < 1e-11 * abs(Ev)
    assert abs(trial.variational_energy(ham) - Ev) < 1e-11 * abs(Ev)
    assert abs(Ev.imag) < 1e-12 * abs(Ev)


def test_determinant_matrix_elements_against_fock_space():
    """<A|B> and <A|H|B> by Loewdin's rules against Fock-space vectors, for generic pairs and for
    pairs whose overlap matrix loses rank 1, 2 (same spin and opposite spins) and 3 (zero by
    the two-body rank of H), each occupied space also mixed by a random invertible matrix so
    the singular values and rotations are not trivial.  Dropping the exchange term or a spin
    block of the integrals fails the rank-2 cases."""
    rng = np.random.default_rng(31)
    M, nch = 5, 4
    h, L, _ = syn.make_hamiltonian(M, nch, rng)
    ham = O.Hamiltonian(h=h, L=L, E0=0.4)
    fs = FockSpace(M, 2, 2)
    H = fs.hamiltonian(h, four_index_from_cholesky(L), ham.E0)
    I = np.eye(M)
    pairs = [((crandn(rng, M, 2), crandn(rng, M, 2)), (crandn(rng, M, 2), crandn(rng, M, 2)))]
    for ua, da, ub, db in [([0, 1], [0, 1], [0, 1], [0, 1]),     # same determinant
                           ([0, 1], [0, 1], [0, 2], [0, 1]),     # single excitation
                           ([0, 1], [0, 1], [2, 3], [0, 1]),     # same-spin double
                           ([0, 1], [0, 1], [0, 2], [1, 3]),     # opposite-spin double
                           ([0, 1], [0, 1], [2, 3], [2, 4]),     # quadruple: zero
                           ([0, 1], [0, 1], [2, 3], [0, 4])]:    # triple: zero
        R = [crandn(rng, 2, 2) for _ in range(4)]
        pairs.append(((I[:, ua] @ R[0], I[:, da] @ R[1]), (I[:, ub] @ R[2], I[:, db] @ R[3])))
    for A, B in pairs:
        S, HAB = determinant_matrix_elements(ham, A, B)
        va, vb = fs.slater_vector(*A), fs.slater_vector(*B)
        Sref, Href = np.vdot(va, vb), np.vdot(va, H @ vb)
        scale = np.linalg.norm(va) * np.linalg.norm(vb)
        assert abs(S - Sref) < 1e-12 * scale
        assert abs(HAB - Href) < 1e-12 * scale * np.linalg.norm(H, 2)


def test_one_and_repeated_determinants_reduce_to_the_single_determinant():
    ham, trial, Phi, _ = system(4)
    D = trial.dets[1]
    E1, t1, _ = O.local_energy(ham, D, Phi)
    ld = sum(O.log_det(O.overlap_matrix(D[s], Phi[s])) for s in range(2))
    for tr, cs in ((MSDTrial([D], [2.0 - 1.0j]), 2.0 + 1.0j), (MSDTrial([D, D], [0.3 + 0.2j, 1.1 - 0.7j]), 1.4 + 0.5j)):
        E, t = tr.local_energy(ham, Phi)
        assert np.max(np.abs(E - E1)) < 1e-12 * np.max(np.abs(E1))
        assert np.max(np.abs(t - t1)) < 1e-12 * np.max(np.abs(t1))
        assert np.max(np.abs(np.exp(tr.log_overlap(Phi) - ld) - cs)) < 1e-12
    E_T = O.local_energy(ham, D, [D[0][None], D[1][None]])[0][0]
    assert abs(MSDTrial([D], [0.5j]).energy_shift(ham) - E_T) < 1e-12 * abs(E_T)


def test_regauged_expansion_is_the_same_state():
    ham, trial, Phi, rng = system(5)
    dets, c = [], []
    for cI, (Du, Dd) in zip(trial.c, trial.dets):
        Ru = crandn(rng, 2, 2) + 2 * np.eye(2)
        Rd = crandn(rng, 2, 2) + 2 * np.eye(2)
        dets.append((Du @ Ru, Dd @ Rd))
        c.append(cI / (np.linalg.det(Ru) * np.linalg.det(Rd)))
    g = MSDTrial(dets, c)
    E, t = trial.local_energy(ham, Phi)
    Eg, tg = g.local_energy(ham, Phi)
    assert np.max(np.abs(Eg - E)) < 1e-11 * np.max(np.abs(E))
    assert np.max(np.abs(tg - t)) < 1e-11 * np.max(np.abs(t))
    assert np.max(np.abs(np.exp(g.log_overlap(Phi) - trial.log_overlap(Phi)) - 1)) < 1e-11
    assert abs(g.energy_shift(ham) - trial.energy_shift(ham)) < 1e-11 * abs(trial.energy_shift(ham))
    # negative control: forgetting the determinant factor changes the state
    bad = MSDTrial(dets, trial.c)
    assert np.max(np.abs(bad.local_energy(ham, Phi)[0] - E)) > 1e-6


def test_phaseless_run_with_an_expansion():
    rng = np.random.default_rng(8)
    M, N, nch = 6, 2, 8
    h, L, E0 = syn.make_hamiltonian(M, nch, rng)
    ham = O.Hamiltonian(h=h, L=L, E0=E0)
    Psi = syn.make_trial(h, N, N)
    p = O.Params(tau=0.01, k_taylor=6, k_qr=2)
    x = rng.standard_normal((5, 4, nch))
    single = O.run(ham, Psi, 4, x, p)
    one = O.run(ham, MSDTrial([Psi], [1.0]), 4, x, p)
    assert np.max(np.abs(np.array(one["E_mix"]) - np.array(single["E_mix"]))) < 1e-12
    # a second, non-orthogonal determinant: the trial's second orbital rotated towards the third
    _, v = np.linalg.eigh(h)
    D2 = np.stack([v[:, 0], np.cos(0.4) * v[:, 1] + np.sin(0.4) * v[:, 2]], axis=1)
    tr = MSDTrial([Psi, (D2, D2)], [1.0, 0.2])
    out = O.run(ham, tr, 4, x, p)
    assert np.all(np.isfinite(np.array(out["E_mix"])))
    assert np.all(out["walkers"].w > 0)
    assert abs(out["E_T"] - tr.energy_shift(ham).real) == 0.0


def test_exact_ground_state_expansion_has_zero_variance_local_energy():
    """Two electrons (one per spin): the FCI ground state is exactly sum_ij C_ij |i up, j dn>, an
    orthogonal expansion over M^2 determinants.  With it as the trial, H|psi_T> = E|psi_T>, so
    the mixed local energy equals E_FCI at any walker (generic walkers overlap every
    determinant); the force-bias traces equal the Fock-space mixed estimates of every L_n.
    The energy shift E_T skips the exactly orthogonal pairs of such an expansion (the oracle's
    stated reading: it is a shift there, not the variational energy), so it equals the
    diagonal part; the variational energy, from every pair's matrix element, is E_FCI."""
    rng = np.random.default_rng(12)
    M, nch = 4, 5
    h, L, _ = syn.make_hamiltonian(M, nch, rng)
    ham = O.Hamiltonian(h=h, L=L, E0=0.2)
    fs = FockSpace(M, 1, 1)
    H = fs.hamiltonian(h, four_index_from_cholesky(L), ham.E0)
    e, V = np.linalg.eigh(H)
    I = np.eye(M)
    dets, c = [], []
    for i in range(M):
        for j in range(M):
            D = (I[:, [i]], I[:, [j]])
            dets.append(D)
            c.append(np.vdot(fs.slater_vector(*D), V[:, 0]))
    trial = MSDTrial(dets, c)
    assert np.max(np.abs(fock_vector(fs, trial) - V[:, 0])) < 1e-12
    Phi = [crandn(rng, 5, M, 1), crandn(rng, 5, M, 1)]
    E, t = trial.local_energy(ham, Phi)
    assert np.max(np.abs(E - e[0])) < 1e-10 * abs(e[0])
    diag = sum(abs(cI) ** 2 * np.vdot(fs.slater_vector(*D), H @ fs.slater_vector(*D)) for cI, D in zip(c, dets))
    assert abs(trial.energy_shift(ham) - diag / np.sum(np.abs(c) ** 2)) < 1e-12 * abs(e[0])
    assert abs(trial.variational_energy(ham) - e[0]) < 1e-10 * abs(e[0])
    vp = V[:, 0]
    for w in range(5):
        vf = fs.slater_vector(Phi[0][w], Phi[1][w])
        ov = np.vdot(vp, vf)
        for n in range(nch):
            assert abs(t[w, n] - np.vdot(vp, fs.one_body_operator(L[n]) @ vf) / ov) < 1e-10
