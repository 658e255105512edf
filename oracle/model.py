"""FP64 oracle of the two neural-network potentials (test infrastructure only).

The paper runs a large foundation model and a distilled 3.5 A model (section
"Neural Network Architectures") whose hyperparameters live in its missing
Supporting Information. Both are stood in for by one invariant
message-passing architecture, defined here as plainly as possible:

    h0_i   = A[Z_i]
    layer l:  u_i   = h_i W_in
              w_ij  = fc(d_ij) * ( SiLU(e(d_ij) W1 + b1) W2 + b2 )
              m_i   = sum_{j in N(i)} w_ij * u_j            (elementwise)
              h_i  <- h_i + SiLU(m_i U1 + c1) U2 + c2
    E_i    = SiLU(h_i R1 + d1) . R2 + d2 + e0[Z_i]
             + (1/2) sum_{j in N(i)} a exp(-d_ij / rho) fc(d_ij; r_rep)
    E      = sum_i E_i                   (per independent system)

    e_k(d) = sqrt(2/rc) sin(k pi d / rc) / d,  k = 1..K   (Bessel basis)
    fc(d)  = (cos(pi d / rc) + 1) / 2 for d < rc, else 0  (cosine cutoff)
    SiLU(a) = a / (1 + exp(-a))

The last term is a short-range pair repulsion (a, rho, r_rep <= rc fixed, not
trained): random-init networks have no repulsive core, which the paper's
trained models do have; the same term in both models cancels in F - F_small.

N(i) is the set of j != i with |r_ij|^2 < rc^2 (strict, FP64), where r_ij is
the minimum-image difference x_j - x_i - L rint((x_j - x_i) / L) in a periodic
cubic box of edge L, or x_j - x_i without periodicity; atoms of different
systems never interact. Forces are F = -dE/dx (the quantity Algorithm 1
consumes); the distillation losses are the force-matching mean square error
and its energy-and-force extension of the knowledge-distillation step
(section "Training procedures"), optimised by Adam.

The derivatives are taken by reverse-mode automatic differentiation of the
energy written above (a library primitive computing the exact derivative);
finite-difference tests pin them independently.
"""
from __future__ import annotations

import math
from typing import NamedTuple, Sequence

import numpy as np
import torch

DT = torch.float64


class Spec(NamedTuple):
    """Architecture: cutoff (A), K radial functions, Lr layers, F features,
    S species; pair repulsion amplitude (eV), decay length and cutoff (A)."""

    cutoff: float
    n_radial: int
    n_layers: int
    n_feat: int
    n_species: int
    rep_a: float = 0.0
    rep_rho: float = 1.0
    rep_cutoff: float = 0.0


def spec_of(obj) -> Spec:
    return Spec(float(obj.cutoff), int(obj.n_radial), int(obj.n_layers),
                int(obj.n_feat), int(obj.n_species), float(getattr(obj, "rep_a", 0.0)),
                float(getattr(obj, "rep_rho", 1.0)), float(getattr(obj, "rep_cutoff", 0.0)))


def parse_params(spec: Spec, p) -> dict:
    """Split the flat parameter vector (documented order: A; per layer W_in,
    W1, b1, W2, b2, U1, c1, U2, c2; R1, d1, R2, d2, e0; matrices row-major,
    input index first) into named float64 tensors sharing storage with ``p``.
    """
    if not torch.is_tensor(p):
        p = torch.as_tensor(np.asarray(p, dtype=np.float64))
    S, F, K = spec.n_species, spec.n_feat, spec.n_radial
    need = S * F + spec.n_layers * (4 * F * F + K * F + 4 * F) + F * F + 2 * F + 1 + S
    if p.numel() != need:
        raise ValueError(f"parameter vector has {p.numel()} entries, layout needs {need}")
    out = {"layers": []}
    pos = 0

    def nxt(*shape):
        nonlocal pos
        n = 1
        for s in shape:
            n *= s
        t = p[pos:pos + n].reshape(shape)
        pos += n
        return t

    out["A"] = nxt(S, F)
    for _ in range(spec.n_layers):
        lay = {}
        lay["W_in"] = nxt(F, F)
        lay["W1"] = nxt(K, F)
        lay["b1"] = nxt(F)
        lay["W2"] = nxt(F, F)
        lay["b2"] = nxt(F)
        lay["U1"] = nxt(F, F)
        lay["c1"] = nxt(F)
        lay["U2"] = nxt(F, F)
        lay["c2"] = nxt(F)
        out["layers"].append(lay)
    out["R1"] = nxt(F, F)
    out["d1"] = nxt(F)
    out["R2"] = nxt(F)
    out["d2"] = nxt(1)
    out["e0"] = nxt(S)
    assert pos == need
    return out


# --------------------------------------------------------------------------
# Neighbour pairs: brute force over all pairs of each system
# --------------------------------------------------------------------------

def _system_ids(atom_offset, n):
    off = np.asarray(atom_offset, dtype=np.int64)
    sid = np.zeros(n, dtype=np.int64)
    for s in range(len(off) - 1):
        sid[off[s]:off[s + 1]] = s
    return sid


def pair_list(x, atom_offset, box, cutoff, chunk: int = 1024):
    """All directed pairs (i, j), j != i, of the same system with
    |r_ij|^2 < cutoff^2, sorted by i then j.

    r_ij is taken in float64 as dx = x_j - x_i, then (periodic) dx - L *
    rint(dx / L), and |r|^2 = (dx*dx + dy*dy) + dz*dz, each operation rounded
    separately (no fused multiply-add). Returns two int64 numpy arrays.
    """
    x = torch.as_tensor(np.asarray(x, dtype=np.float64))
    off = np.asarray(atom_offset, dtype=np.int64)
    box = np.asarray(box, dtype=np.float64)
    rc2 = float(cutoff) * float(cutoff)
    I, J = [], []
    for s in range(len(off) - 1):
        a, b = int(off[s]), int(off[s + 1])
        xs = x[a:b]
        L = float(box[s])
        if L > 0 and L < 2.0 * cutoff:
            raise ValueError("periodic box edge must be at least twice the cutoff")
        n = b - a
        for c0 in range(0, n, chunk):
            c1 = min(n, c0 + chunk)
            dx = xs[None, :, :] - xs[c0:c1, None, :]          # x_j - x_i
            if L > 0:
                dx = dx - L * torch.round(dx / L)             # round-half-even
            d2 = (dx[..., 0] * dx[..., 0] + dx[..., 1] * dx[..., 1]) + dx[..., 2] * dx[..., 2]
            mask = d2 < rc2
            idx = torch.arange(c0, c1)
            mask[idx - c0, idx] = False                        # no self pairs
            ii, jj = torch.nonzero(mask, as_tuple=True)
            I.append((ii + c0 + a).numpy())
            J.append((jj + a).numpy())
    if not I:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    I = np.concatenate(I)
    J = np.concatenate(J)
    order = np.lexsort((J, I))
    return I[order], J[order]


def pair_row(x, i, atom_offset, box, cutoff):
    """Row i of the pair list (sorted j), by the same FP64 expression as
    ``pair_list``; for checking sampled rows of systems too large for the
    full O(N^2) list."""
    x = np.asarray(x, dtype=np.float64)
    off = np.asarray(atom_offset, dtype=np.int64)
    s = int(np.searchsorted(off, i, side="right") - 1)
    a, b = int(off[s]), int(off[s + 1])
    L = float(np.asarray(box, dtype=np.float64)[s])
    dx = torch.as_tensor(x[a:b]) - torch.as_tensor(x[i])[None, :]
    if L > 0:
        dx = dx - L * torch.round(dx / L)
    d2 = (dx[:, 0] * dx[:, 0] + dx[:, 1] * dx[:, 1]) + dx[:, 2] * dx[:, 2]
    mask = d2 < float(cutoff) * float(cutoff)
    mask[i - a] = False
    return (torch.nonzero(mask)[:, 0] + a).numpy()


def pair_vectors(x, i, j, atom_offset, box):
    """Minimum-image r_ij = x_j - x_i for the given pairs (differentiable in
    x; the integer image shift carries no derivative)."""
    sid = torch.as_tensor(_system_ids(atom_offset, x.shape[0]))
    L = torch.as_tensor(np.asarray(box, dtype=np.float64))[sid[i]]
    i = torch.as_tensor(i)
    j = torch.as_tensor(j)
    r = x[j] - x[i]
    per = (L > 0)
    if bool(per.any()):
        Lc = torch.where(per, L, torch.ones_like(L))[:, None]
        shift = torch.where(per[:, None], Lc * torch.round(r.detach() / Lc), torch.zeros_like(r))
        r = r - shift
    return r


# --------------------------------------------------------------------------
# Radial basis, cutoff, activation
# --------------------------------------------------------------------------

def bessel_basis(d, cutoff: float, K: int):
    """e_k(d) = sqrt(2/rc) sin(k pi d / rc) / d for k = 1..K; [E, K]."""
    k = torch.arange(1, K + 1, dtype=DT)
    return math.sqrt(2.0 / cutoff) * torch.sin(k[None, :] * math.pi * d[:, None] / cutoff) / d[:, None]


def cosine_cutoff(d, cutoff: float):
    """fc(d) = (cos(pi d / rc) + 1) / 2 inside the cutoff, 0 outside."""
    inside = 0.5 * (torch.cos(math.pi * d / cutoff) + 1.0)
    return torch.where(d < cutoff, inside, torch.zeros_like(d))


def silu(a):
    return a * torch.sigmoid(a)


# --------------------------------------------------------------------------
# Energy, forces, virial
# --------------------------------------------------------------------------

def atomic_energies_from_pairs(spec: Spec, P: dict, species, i, j, r):
    """E_i for every atom given the pair list and pair vectors r_ij."""
    n = species.shape[0]
    i = torch.as_tensor(i)
    j = torch.as_tensor(j)
    species = torch.as_tensor(np.asarray(species, dtype=np.int64))
    d = torch.sqrt((r * r).sum(dim=1))
    e = bessel_basis(d, spec.cutoff, spec.n_radial)
    fc = cosine_cutoff(d, spec.cutoff)
    h = P["A"][species]
    for lay in P["layers"]:
        u = h @ lay["W_in"]
        phi = silu(e @ lay["W1"] + lay["b1"]) @ lay["W2"] + lay["b2"]
        w = fc[:, None] * phi
        m = torch.zeros(n, spec.n_feat, dtype=DT).index_add(0, i, w * u[j])
        h = h + silu(m @ lay["U1"] + lay["c1"]) @ lay["U2"] + lay["c2"]
    Ei = silu(h @ P["R1"] + P["d1"]) @ P["R2"] + P["d2"][0] + P["e0"][species]
    if spec.rep_a != 0.0 and spec.rep_cutoff > 0.0:
        phi = spec.rep_a * torch.exp(-d / spec.rep_rho) * cosine_cutoff(d, spec.rep_cutoff)
        Ei = Ei + 0.5 * torch.zeros(n, dtype=DT).index_add(0, i, phi)
    return Ei


def energy(spec: Spec, params, x, species, atom_offset, box, pairs=None):
    """Per-system potential energy [n_systems] (eV), float64 tensor."""
    P = parse_params(spec, params)
    x = torch.as_tensor(x) if torch.is_tensor(x) else torch.as_tensor(np.asarray(x, dtype=np.float64))
    if pairs is None:
        pairs = pair_list(x.detach().numpy(), atom_offset, box, spec.cutoff)
    i, j = pairs
    r = pair_vectors(x, i, j, atom_offset, box)
    Ei = atomic_energies_from_pairs(spec, P, species, i, j, r)
    sid = torch.as_tensor(_system_ids(atom_offset, x.shape[0]))
    return torch.zeros(len(atom_offset) - 1, dtype=DT).index_add(0, sid, Ei)


def energy_forces(spec: Spec, params, x, species, atom_offset, box, pairs=None):
    """(E [n_systems], F [N, 3]) as numpy float64, F = -dE/dx."""
    xt = torch.tensor(np.asarray(x, dtype=np.float64), requires_grad=True)
    E = energy(spec, params, xt, species, atom_offset, box, pairs)
    (g,) = torch.autograd.grad(E.sum(), xt)
    return E.detach().numpy(), (-g).numpy()


def virial(spec: Spec, params, x, species, atom_offset, box, pairs=None):
    """Per-system virial W_ab = -dE/d(eps_ab) [n_systems, 3, 3] under the
    homogeneous deformation r_ij -> r_ij (I + eps)^T of every pair vector,
    i.e. W = -sum_pairs r_ij (x) dE/dr_ij. For a periodic box this is the
    strain derivative with the image assignment held fixed."""
    P = parse_params(spec, params)
    xt = torch.as_tensor(np.asarray(x, dtype=np.float64))
    if pairs is None:
        pairs = pair_list(x, atom_offset, box, spec.cutoff)
    i, j = pairs
    ns = len(atom_offset) - 1
    sid = torch.as_tensor(_system_ids(atom_offset, xt.shape[0]))
    eps = torch.zeros(ns, 3, 3, dtype=DT, requires_grad=True)
    r0 = pair_vectors(xt, i, j, atom_offset, box)
    def_ = torch.eye(3, dtype=DT)[None] + eps                 # [ns, 3, 3]
    r = torch.einsum("eab,eb->ea", def_[sid[torch.as_tensor(i)]], r0)
    Ei = atomic_energies_from_pairs(spec, P, species, i, j, r)
    E = torch.zeros(ns, dtype=DT).index_add(0, sid, Ei)
    (g,) = torch.autograd.grad(E.sum(), eps)
    return (-g).numpy()


def strained_energy(spec: Spec, params, x, species, atom_offset, box, eps, pairs):
    """Energy with every pair vector deformed by (I + eps); for the virial's
    finite-difference pin."""
    P = parse_params(spec, params)
    xt = torch.as_tensor(np.asarray(x, dtype=np.float64))
    i, j = pairs
    r = pair_vectors(xt, i, j, atom_offset, box) @ (torch.eye(3, dtype=DT) + torch.as_tensor(eps)).T
    Ei = atomic_energies_from_pairs(spec, P, species, i, j, r)
    return float(Ei.sum())


# --------------------------------------------------------------------------
# Force-matching distillation loss and its parameter gradient
# --------------------------------------------------------------------------

def force_matching_loss(spec: Spec, params, frames, species, atom_offset, box,
                        f_ref, create_graph: bool = False):
    """L(theta) = 1/(3 N M) sum_m sum_i |F_i(theta; x_m) - F_ref_{m,i}|^2 over
    M frames, with F = -dE/dx of the model with parameters theta. Returns a
    scalar tensor (differentiable in ``params`` if it is a tensor requiring
    grad and ``create_graph``)."""
    frames = np.asarray(frames, dtype=np.float64)
    f_ref = np.asarray(f_ref, dtype=np.float64)
    M, N = frames.shape[0], frames.shape[1]
    total = torch.zeros((), dtype=DT)
    for m in range(M):
        xt = torch.tensor(frames[m], requires_grad=True)
        E = energy(spec, params, xt, species, atom_offset, box)
        (g,) = torch.autograd.grad(E.sum(), xt, create_graph=create_graph)
        F = -g
        total = total + ((F - torch.as_tensor(f_ref[m])) ** 2).sum()
    return total / (3.0 * N * M)


def force_matching_grad(spec: Spec, params, frames, species, atom_offset, box, f_ref):
    """(L, dL/dtheta) as (float, numpy float64 [n_params]); the gradient goes
    through the forces, i.e. second derivatives of the energy."""
    th = torch.tensor(np.asarray(params, dtype=np.float64), requires_grad=True)
    L = force_matching_loss(spec, th, frames, species, atom_offset, box, f_ref, create_graph=True)
    (g,) = torch.autograd.grad(L, th)
    return float(L.detach()), g.numpy()


def distill_loss(spec: Spec, params, frames, species, atom_offset, box, f_ref, e_ref, lambda_e: float,
                 create_graph: bool = False):
    """Energy and force distillation loss over M frames (the small model fit
    to the large model's energies and forces of MD frames, section "Training
    procedures"):
        L = 1/M sum_m [ lambda_e ((E_m - E_ref,m) / N)^2
                        + 1/(3 N) sum_i |F_i(x_m) - F_ref,m,i|^2 ],
    E_m the frame's energy summed over its systems, N its atom count. With
    lambda_e = 0 it is ``force_matching_loss``."""
    frames = np.asarray(frames, dtype=np.float64)
    f_ref = np.asarray(f_ref, dtype=np.float64)
    e_ref = np.asarray(e_ref, dtype=np.float64).reshape(-1)
    M, N = frames.shape[0], frames.shape[1]
    total = torch.zeros((), dtype=DT)
    for m in range(M):
        xt = torch.tensor(frames[m], requires_grad=True)
        E = energy(spec, params, xt, species, atom_offset, box).sum()
        (g,) = torch.autograd.grad(E, xt, create_graph=create_graph)
        total = total + ((-g - torch.as_tensor(f_ref[m])) ** 2).sum() / (3.0 * N)
        total = total + lambda_e * ((E - float(e_ref[m])) / N) ** 2
    return total / M


def distill_grad(spec: Spec, params, frames, species, atom_offset, box, f_ref, e_ref, lambda_e: float):
    """(L, dL/dtheta) of ``distill_loss`` as (float, numpy float64 [n_params])."""
    th = torch.tensor(np.asarray(params, dtype=np.float64), requires_grad=True)
    L = distill_loss(spec, th, frames, species, atom_offset, box, f_ref, e_ref, lambda_e, create_graph=True)
    (g,) = torch.autograd.grad(L, th)
    return float(L.detach()), g.numpy()


def adam_step(theta, grad, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """Step t (1-based) of Adam (Kingma and Ba, ICLR 2015, Algorithm 1):
    biased first and second moment estimates, their bias corrections, and
    the update theta - lr m_hat / (sqrt(v_hat) + eps). Returns (theta, m, v)."""
    g = np.asarray(grad, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return np.asarray(theta, dtype=np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps), m, v

