"""FP64 CPU oracle for the derivative of unrolled IRCUR-F.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this
module: only the tests use it.  It shares no code with the CUDA library.

The map differentiated is Algorithm 1 with fixed index sets I, J (IRCUR-F,
Sec. 3.4) run for exactly T iterations from L_0 = 0, with the thresholds
zeta_{k+1} = gamma^k zeta_0 held fixed:

    for k = 0 .. T-1:
        R_{k+1} = D(I,:) - T_zeta_k(D(I,:) - L_k(I,:))          (Phase I, Sec. 3.2)
        C_{k+1} = D(:,J) - T_zeta_k(D(:,J) - L_k(:,J))
        U_{k+1} = H_r([D - S_{k+1}](I,J))                         (Phase II, Sec. 3.1)
        L_{k+1} = C_{k+1} U_{k+1}^+ R_{k+1}                        (Thm 1)
    outputs: L = L_T and S = T_{zeta_T}(D - L_T), zeta_T = gamma^T zeta_0.

It is written here in plain PyTorch CPU operations in FP64 (dense L_k, the
literal formulas above) and differentiated by reverse-mode automatic
differentiation: the hard-thresholding operator contributes its almost-
everywhere derivative (the keep mask) and the rank-r truncated SVD the
standard SVD derivative through torch.linalg.svd (a library primitive), which
needs distinct singular values and sigma_r > sigma_{r+1}.  zeta_0 enters as a
constant: when it is max|D| its dependence on D changes only where the masks
switch, a set of measure zero, so the derivative there is zero.
"""

from __future__ import annotations

import numpy as np
import torch


def _ht(X, zeta):
    """T_zeta(X): keep the entries with |X_ij| > zeta (Sec. 3.2)."""
    return X * (X.abs() > zeta).to(X.dtype)


def unrolled_forward(D, I, J, r, zeta0, gamma, T, final_keep=None):
    """(L_T, S_T) of the T-step fixed-index map above (torch FP64 tensors).

    final_keep (optional boolean n1 x n2 array) replaces the decisions
    |D - L_T| > zeta_T of the last threshold: the tie reading of T_zeta
    (Sec. 3.2), where an entry within rounding of zeta may go either way and a
    caller supplies the side another evaluation took.  The caller checks that
    it differs from the FP64 decisions only at such ties."""
    I = torch.as_tensor(np.asarray(I, np.int64))
    J = torch.as_tensor(np.asarray(J, np.int64))
    n1, n2 = D.shape
    L = torch.zeros(n1, n2, dtype=D.dtype)
    zeta = float(zeta0)
    for _ in range(T):
        D_rows, D_cols = D[I, :], D[:, J]
        R = D_rows - _ht(D_rows - L[I, :], zeta)
        C = D_cols - _ht(D_cols - L[:, J], zeta)
        core = R[:, J]  # = C[I, :]
        W, s, Vh = torch.linalg.svd(core, full_matrices=False)
        U_pinv = Vh[:r, :].T @ torch.diag(1.0 / s[:r]) @ W[:, :r].T
        L = C @ U_pinv @ R
        zeta = zeta * gamma
    if final_keep is None:
        S = _ht(D - L, zeta)
    else:
        S = (D - L) * torch.as_tensor(np.asarray(final_keep, bool)).to(D.dtype)
    return L, S


def unrolled_vjp(D, I, J, r, zeta0, gamma, T, dL=None, dS=None, final_keep=None):
    """dD = d<dL, L_T> / dD + d<dS, S_T> / dD at D (numpy FP64 in and out);
    final_keep as in unrolled_forward."""
    Dt = torch.tensor(np.asarray(D, np.float64), requires_grad=True)
    L, S = unrolled_forward(Dt, I, J, r, zeta0, gamma, T, final_keep)
    loss = torch.zeros((), dtype=torch.float64)
    if dL is not None:
        loss = loss + (torch.as_tensor(np.asarray(dL, np.float64)) * L).sum()
    if dS is not None:
        loss = loss + (torch.as_tensor(np.asarray(dS, np.float64)) * S).sum()
    loss.backward()
    return Dt.grad.numpy().copy()


def unrolled_outputs(D, I, J, r, zeta0, gamma, T):
    """(L_T, S_T) as numpy FP64 arrays."""
    with torch.no_grad():
        L, S = unrolled_forward(torch.tensor(np.asarray(D, np.float64)), I, J, r, zeta0, gamma, T)
    return L.numpy(), S.numpy()


def masks(D, I, J, r, zeta0, gamma, T):
    """Keep masks of every thresholding step (for checking that a finite-difference
    step stays inside one smooth piece of the map)."""
    I = np.asarray(I, np.int64)
    J = np.asarray(J, np.int64)
    with torch.no_grad():
        Dt = torch.tensor(np.asarray(D, np.float64))
        n1, n2 = Dt.shape
        L = torch.zeros(n1, n2, dtype=torch.float64)
        zeta = float(zeta0)
        out = []
        for _ in range(T):
            Rr = Dt[I, :] - L[I, :]
            Cc = Dt[:, J] - L[:, J]
            out += [(Rr.abs() > zeta).numpy(), (Cc.abs() > zeta).numpy()]
            R = Dt[I, :] - _ht(Rr, zeta)
            C = Dt[:, J] - _ht(Cc, zeta)
            W, s, Vh = torch.linalg.svd(R[:, J], full_matrices=False)
            L = C @ (Vh[:r, :].T @ torch.diag(1.0 / s[:r]) @ W[:, :r].T) @ R
            zeta *= gamma
        out.append(((Dt - L).abs() > zeta).numpy())
    return out
