"""Algorithmic operation counts of the stabilised method (real flops; a complex multiply-add
counts 8, a real x complex multiply-add 4).  Padding and repeated work are not counted; the
same counts are used for every path (CPU oracle, FP64 GPU, mixed GPU).

Per configuration with n = Nx, blocks nb = Nt / n_stab:
  slice products  (Section 7 products, Section 9 blocking):  4 n^3 per slice  (E real)
  QR re-orthogonalisation per block: factor 16/3 n^3 + form Q 16/3 n^3 + T update 4 n^3
  assembly (Section 7 steps 4-6, scale separated): LU 8/3 n^3 + solve 8 n^3
  force (Section 4 response, Section 5.3 pre/suffix): right products 4 n^3 per slice for all
    but the first block, wraps 8 n^3 per slice (all slices but the nb block boundaries), one QR
    (44/3 n^3) and one boundary Green's function (2 GEMMs 16 n^3 + LU 8/3 + solve 8 +
    product 8 = 104/3 n^3) per interior block boundary (nb - 1 of each).
  unequal-time G(tau, 0) (Section 4.2, Section 7 steps 7-9): the chains of the force, a boundary
    solve per interior boundary (104/3 n^3; 16 n^3 more when G_t is formed beside it: a second
    right-hand side and product), and one real x complex product 4 n^3 per propagated slice.
  response traces tr(O G_r): 4 n^2 per slice (real O, complex G) on top of the force's G_r.
  product-form slices (Sections 8-9, q entries per row of K, nf factors): per slice and matrix
    element 4q + 8 per factor (q real x complex multiply-adds, one complex multiply-add by
    gamma_k) and 6 (q + 1) for the field phase folded into the first factor.
"""
from __future__ import annotations


def fwd_flops(nx: int, nt: int, n_stab: int) -> dict:
    n3 = float(nx) ** 3
    nb = nt // n_stab
    slices = 4.0 * n3 * nt
    qr = (44.0 / 3.0) * n3 * nb
    asm = (32.0 / 3.0) * n3
    return {"slices": slices, "qr": qr, "assembly": asm, "total": slices + qr + asm}


def force_flops(nx: int, nt: int, n_stab: int) -> dict:
    """Forward pass (with checkpoints) plus the adjoint sweep."""
    f = fwd_flops(nx, nt, n_stab)
    n3 = float(nx) ** 3
    nb = nt // n_stab
    right = 4.0 * n3 * (nt - n_stab)
    wraps = 8.0 * n3 * (nt - nb)
    qr = (44.0 / 3.0) * n3 * (nb - 1)
    boundary = (104.0 / 3.0) * n3 * (nb - 1)
    bwd = right + wraps + qr + boundary
    return {"forward": f["total"], "backward": bwd, "total": f["total"] + bwd,
            "slices_and_wraps": f["slices"] + right + wraps,
            "per_block_fp64": f["qr"] + f["assembly"] + qr + boundary}


def force_phase_flops(nx: int, nt: int, n_stab: int, mixed: bool) -> dict:
    """Algorithmic work of the three launches of the force, split by arithmetic pipe.

    A (chains): forward slices 4n^3 Nt and QRs (44/3 n^3 each, nb of them), backward right
       products 4n^3 (Nt - n_stab) and QRs (nb - 1), the assembly (32/3 n^3);
    B (boundary Green's functions): (104/3) n^3 for each of the nb - 1 interior boundaries;
    C (wraps): 8 n^3 for each of the Nt - nb wrapped slices.
    With mixed=True the slice/right products and wraps are tensor-core work, else FP64."""
    n3 = float(nx) ** 3
    nb = nt // n_stab
    a_prod = 4 * n3 * nt + 4 * n3 * (nt - n_stab)
    a_qr = (44.0 / 3.0) * n3 * (2 * nb - 1) + (32.0 / 3.0) * n3
    b = (104.0 / 3.0) * n3 * (nb - 1)
    c = 8 * n3 * (nt - nb)
    if mixed:
        return {"A": {"fp64": a_qr, "tensor": a_prod}, "B": {"fp64": b, "tensor": 0.0},
                "C": {"fp64": 0.0, "tensor": c}}
    return {"A": {"fp64": a_qr + a_prod, "tensor": 0.0}, "B": {"fp64": b, "tensor": 0.0},
            "C": {"fp64": c, "tensor": 0.0}}


def gtau_phase_flops(nx: int, nt: int, n_stab: int, mixed: bool) -> dict:
    """The three launches of log det + G(tau, 0) (no force): chains as for the force, boundary
    solves for G((b-1) n_stab, 0), and the propagation inside the blocks (FP64 in every mode)."""
    base = force_phase_flops(nx, nt, n_stab, mixed)
    n3 = float(nx) ** 3
    nb = nt // n_stab
    return {"A": base["A"], "B": {"fp64": (104.0 / 3.0) * n3 * (nb - 1), "tensor": 0.0},
            "C": {"fp64": 4 * n3 * (nt - nb), "tensor": 0.0}}


def response_phase_flops(nx: int, nt: int, n_stab: int, mixed: bool) -> dict:
    """log det + response traces: the force's launches plus 4 n^2 per slice for the traces
    (FP64 in the FP64 path; FP32 CUDA-core work in the mixed epilogue, not counted there)."""
    base = force_phase_flops(nx, nt, n_stab, mixed)
    if not mixed:
        base["C"] = {"fp64": base["C"]["fp64"] + 4.0 * nx * nx * nt, "tensor": 0.0}
    return base


def sparse_fwd_flops(nx: int, nt: int, n_stab: int, q: int, nfac: int) -> dict:
    """log det/G with the product-form slices: the slices above, QR and assembly as fwd_flops."""
    n2 = float(nx) ** 2
    slices = (nfac * (4.0 * q + 8.0) + 6.0 * (q + 1)) * n2 * nt
    f = fwd_flops(nx, nt, n_stab)
    return {"slices": slices, "qr": f["qr"], "assembly": f["assembly"],
            "total": slices + f["qr"] + f["assembly"]}
