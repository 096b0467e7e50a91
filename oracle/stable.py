"""The stabilised dense small-volume method of Section 7, in numpy/scipy FP64.

Representation (Eq. def_matrix_as_product): a matrix is kept as X diag(D) Y^{-1} with X unitary,
D > 0 diagonal (spanning many orders of magnitude) and Y^{-1} =: T of order-one entries, never
contracted.  Multiplying slices onto it and re-factorising follows Eqs. prod_2_mat_stab ..
res_2_mat_stab: the contracted middle factor is QR-decomposed, X' = Q, D = |diag R|,
Y'^{-1} = D^{-1} R.  As proposed in Section 9, the QR is done only every n_stab slices; in
between, slices are multiplied onto X directly.

Readings of the paper used here (each is listed in the design notes):
  * Pivoting.  Section 7 asks for D sorted by magnitude; a plain QR does not give that, so the
    QR uses column pivoting (LAPACK geqp3 via scipy), D = |diag R| and the unit-modulus phases
    of diag R stay in T.
  * Assembly.  Step 4 of Section 7 QR-decomposes 1 + D Y^{-1} X.  With D up to e^{+-200} that
    mixes rows of wildly different scale, so the main assembly splits D = D_b D_s with
    D_b = max(D, 1), D_s = min(D, 1) and uses
        1 + X D T = X D_b (D_b^{-1} X^H + D_s T) =: X D_b C,
        log det(1 + X D T) = log det X + sum log D_b + log det C,
        G = C^{-1} D_b^{-1} X^H.
    The literal step-4..6 form is kept in :func:`assemble_literal` as a small-beta cross-check.
  * Branch.  log det is complex; its imaginary part is returned wrapped to (-pi, pi].
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .plain import slice_matrix


def reorthogonalise(X: np.ndarray, D: np.ndarray, T: np.ndarray):
    """Re-factor X diag(D) T = X' diag(D') T' with a pivoted QR of Z = X diag(D).

    Z Pi = Q R  =>  X diag(D) T = Q R Pi^T T = Q diag(|diag R|) [diag(|diag R|)^{-1} R Pi^T T].
    """
    Z = X * D[None, :]
    Q, R, perm = scipy.linalg.qr(Z, pivoting=True)
    d = np.abs(np.diag(R))
    T_new = (R / d[:, None]) @ T[perm, :]
    return Q, d, T_new


def udt_product(E: np.ndarray, phi: np.ndarray, n_stab: int):
    """B_Nt ... B_1 as (X, D, T), a QR every n_stab slices (the last block may be shorter)."""
    nt, nx = phi.shape
    X = np.eye(nx, dtype=complex)
    D = np.ones(nx)
    T = np.eye(nx, dtype=complex)
    t = 0
    while t < nt:
        for s in range(t, min(t + n_stab, nt)):
            X = slice_matrix(E, phi[s]) @ X
        X, D, T = reorthogonalise(X, D, T)
        t += n_stab
    return X, D, T


def udv_times_udv(later, earlier):
    """Stabilised product of two UDV factors (Section 7): (Xs Ds Ts)(Xa Da Ta) =
    Xs [Ds (Ts Xa)] Da Ta, the bracket times Da re-factored by a pivoted QR, X = Xs Q."""
    Xs, Ds, Ts = later
    Xa, Da, Ta = earlier
    C = Ds[:, None] * (Ts @ Xa)
    Q, d, T_new = reorthogonalise(C, Da, Ta)
    return Xs @ Q, d, T_new


def segmented_product(E: np.ndarray, phi: np.ndarray, n_stab: int, nseg: int):
    """B_Nt ... B_1 from nseg consecutive segments, each a udt_product from the identity, merged
    in time order with udv_times_udv (the same product as udt_product, in another order)."""
    nt = phi.shape[0]
    k = nt // nseg
    segs = [udt_product(E, phi[s * k:(s + 1) * k], n_stab) for s in range(nseg)]
    acc = segs[0]
    for s in range(1, nseg):
        acc = udv_times_udv(segs[s], acc)
    return acc


def assemble(X: np.ndarray, D: np.ndarray, T: np.ndarray):
    """(log det(1 + X D T), (1 + X D T)^{-1}) with the D_b / D_s scale separation."""
    Db = np.maximum(D, 1.0)
    Ds = np.minimum(D, 1.0)
    XH = X.conj().T
    C = XH / Db[:, None] + Ds[:, None] * T
    sx, lx = np.linalg.slogdet(X)
    sc, lc = np.linalg.slogdet(C)
    logdet = (lx + lc + np.sum(np.log(Db))) + 1j * (np.angle(sx) + np.angle(sc))
    G = np.linalg.solve(C, XH / Db[:, None])
    return _wrap(logdet), G


def assemble_literal(X: np.ndarray, D: np.ndarray, T: np.ndarray):
    """Steps 4-6 of Section 7 as printed: QR of 1 + D Y^{-1} X = Qh Dh Rh with diag Rh = 1,
    log det = i arg det Qh + sum log Dh, and G = (X Rh^{-1}) Dh^{-1} (Qh^H X^{-1}).
    No scale separation, so only for moderate beta."""
    nx = X.shape[0]
    A = np.eye(nx) + D[:, None] * (T @ X)
    Q, R = np.linalg.qr(A)
    dh = np.diag(R).copy()
    Rh = R / dh[:, None]
    sq, _ = np.linalg.slogdet(Q)
    logdet = 1j * np.angle(sq) + np.sum(np.log(dh.astype(complex)))
    XRinv = X @ np.linalg.inv(Rh)
    G = XRinv @ np.diag(1.0 / dh) @ (Q.conj().T @ np.linalg.inv(X))
    return _wrap(logdet), G


def logdet_green(E: np.ndarray, phi: np.ndarray, n_stab: int):
    """Stabilised (log det(1 + B_Nt...B_1), (1 + B_Nt...B_1)^{-1})."""
    return assemble(*udt_product(E, phi, n_stab))


def _wrap(z: complex) -> complex:
    im = float(np.angle(np.exp(1j * np.imag(z))))
    if im <= -np.pi:
        im += 2 * np.pi
    return complex(np.real(z), im)
