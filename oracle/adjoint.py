"""FP64 adjoint of the sCOLA forward run (vector-Jacobian products, hand derived).

Test infrastructure (see ``oracle/__init__``).

Entry points: ``final_state_vjp`` turns dL/dx and dL/dp of the final positions and
momenta of a run into dL/dw (w the white noise); ``loss_and_grad`` composes it with the
periodic CIC adjoint for the loss Lval = sum_c (delta_f(c) - delta_t(c))^2 over the
periodic N^3 CIC density of the final positions (Sec. 4.1).  The gradient is assembled
backwards through every step of ``scola.run_scola``:

  delta_f = CIC(x)                      -> lam_x = dCIC/dx^T lam_delta        (weight gradients)
  x = (q + s_n) mod L  (tile particles) -> lam_s(n) = lam_x
  p = p_res + a^2 calH (-dD1/da Psi1 + dD2/da Psi2)  (L+, Eq. 55)
                                        -> lam_p_res = lam_p, lam_Psi1, lam_Psi2
  KDK in reverse (App. B, Eqs. 53-54), per box, with the displacements s_k of
  every force evaluation recomputed forward and kept (checkpoints):
      drift  s_k+1 = s_k + alpha p + d1 Psi1 + d2 Psi2
             -> lam_p += alpha lam_s,  lam_Psi1 += d1 lam_s,  lam_Psi2 += d2 lam_s
      kick   p += kF F(s_k) + k1 Psi1 + k2 Psi2
             -> lam_F = kF lam_p,  lam_Psi1 += k1 lam_p,  lam_Psi2 += k2 lam_p
      force  F(s) = B-bar(grad Phi[delta(s), Phi_BC])  (Sec. 3.4)
             -> lam_s += dF/ds^T lam_F through (i) the interpolation weights,
                (ii) the mesh: lam_G = CIC deposit of lam_F, lam_Phi = -div lam_G,
                lam_delta' = Dirichlet solve of lam_Phi (the Dirichlet Laplacian is
                symmetric), lam_s += d delta/ds^T lam_delta (deposit weights), and
                lam_Phi_BC from the ghost layers and the boundary source of Eq. 62
  L-     s_0 = -D1(a_i) Psi1 + D2(a_i) Psi2 -> lam_Psi1, lam_Psi2
  C.3    Phi_BC = D1(a_K) * trilinear(phi1) -> lam_phi1 (trilinear transpose)
  C.2    Psi = central gradient            -> lam_phi = -div lam_Psi
  A.2    phi2 = Lap^-1 S(phi1), S bilinear in the second derivatives of phi1
         phi1 = Lap^-1 delta_i              (symmetric Fourier operators)
  A.1    delta_i = colour(w)                (real symmetric filter)

Every stencil follows the run's FDA order (2, 4 or 6, Sec. 3.1): the order-n gradient at
the CIC corners and in the LPT stage, the order-n boundary source and Laplacian symbol,
n ghost layers.  Per-tile final scale factors give every box its own coefficients.

Pins (tests/test_oracle_adjoint.py): dot-product identities <J v, u> = <v, J^T u>
for each linear piece, and FP64 central finite differences of the whole loss
along random directions (orders 2, 4, 6; both LPT frames; both KDK factor sets;
per-tile final scale factors), with the adjoint's own forward sweep checked against
the method's run.
"""
import numpy as np

from . import boundary, cosmology, fda, ics, lpt, pm, scola, stats, tiling


# ----------------------------------------------------------------------------- CIC pieces
def _corner_weights(u):
    """i0, and for each of the 8 corners: offsets, weight, d weight / du (per axis)."""
    i0 = np.floor(u).astype(np.int64)
    f = u - i0
    out = []
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                d = np.array([dx, dy, dz])
                w1 = [f[:, a] if d[a] else 1.0 - f[:, a] for a in range(3)]
                g1 = [np.ones_like(f[:, a]) if d[a] else -np.ones_like(f[:, a]) for a in range(3)]
                w = w1[0] * w1[1] * w1[2]
                dw = np.stack([g1[0] * w1[1] * w1[2], w1[0] * g1[1] * w1[2], w1[0] * w1[1] * g1[2]], 1)
                out.append((d, w, dw))
    return i0, out


def periodic_density_vjp(x, L, N, Np, lam_delta):
    """lam_x = d(CIC density on N^3)/dx^T lam_delta  (Sec. 4.1 density, periodic)."""
    d = L / N
    u = np.asarray(x, dtype=np.float64) / d - 0.5
    i0, corners = _corner_weights(u)
    scale = float(N) ** 3 / float(Np) ** 3
    lam = np.zeros_like(u)
    for off, w, dw in corners:
        c = (i0 + off) % N
        v = lam_delta[c[:, 0], c[:, 1], c[:, 2]]
        lam += dw * v[:, None]
    return lam * scale / d


def box_density_vjp(xloc, dg, Ng, Nsc, lam_delta):
    """lam_s = d(B^sCOLA density)/ds^T lam_delta over the interior cells (Sec. 3.4.1)."""
    u = pm.mesh_coordinate(xloc, dg)
    i0, corners = _corner_weights(u)
    lam = np.zeros_like(u)
    inv_nbar = (Ng / Nsc) ** 3
    for off, w, dw in corners:
        c = i0 + off
        inside = np.all((c >= 0) & (c < Ng), axis=1)
        v = np.zeros(len(u))
        v[inside] = lam_delta[c[inside, 0], c[inside, 1], c[inside, 2]]
        lam += dw * v[:, None]
    return lam * inv_nbar / dg


def _shift_add(out, src, a, m, sign):
    """out[c + m e_a] += sign * src[c] (m may be negative; entries shifted out are dropped)."""
    n = src.shape[a]
    dst_sl = [slice(None)] * 3
    src_sl = [slice(None)] * 3
    if m >= 0:
        dst_sl[a], src_sl[a] = slice(m, n), slice(0, n - m)
    else:
        dst_sl[a], src_sl[a] = slice(0, n + m), slice(-m, n)
    out[tuple(dst_sl)] += sign * src[tuple(src_sl)]


def interp_vjp(phi_pad, xloc, dg, lam_F, order=2):
    """VJP of F = interpolate_gradient(phi_pad, x) at FDA order n: returns (lam_x, lam_phi_pad)."""
    P, ng = order, fda.n_ghost(order)
    Ng = phi_pad.shape[0] - 2 * P
    g = fda.gradient_coefficients(order)
    u_raw = pm.mesh_coordinate(xloc, dg)
    u = np.clip(u_raw, -float(ng), float(Ng + ng - 1))
    free = (u == u_raw).astype(np.float64)               # d u / d u_raw (0 where clamped)
    i0 = np.minimum(np.floor(u).astype(np.int64), Ng + ng - 2)
    f = u - i0
    Pp = phi_pad
    lam_x = np.zeros_like(u)
    lam_G = np.zeros((3,) + Pp.shape)                    # adjoint of the gradient mesh
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                d = (dx, dy, dz)
                w1 = [f[:, a] if d[a] else 1.0 - f[:, a] for a in range(3)]
                g1 = [1.0 if d[a] else -1.0 for a in range(3)]
                w = w1[0] * w1[1] * w1[2]
                dw = np.stack([g1[0] * w1[1] * w1[2], w1[0] * g1[1] * w1[2], w1[0] * w1[1] * g1[2]], 1)
                c = [i0[:, a] + d[a] + P for a in range(3)]
                G = np.zeros_like(u)
                for a in range(3):
                    for m, gm in enumerate(g, start=1):
                        cp, cm = list(c), list(c)
                        cp[a], cm[a] = c[a] + m, c[a] - m
                        G[:, a] += gm * (Pp[cp[0], cp[1], cp[2]] - Pp[cm[0], cm[1], cm[2]])
                G /= dg
                # direct term: d w / d u * (G . lam_F)
                lam_x += dw * np.sum(G * lam_F, axis=1)[:, None]
                for a in range(3):
                    np.add.at(lam_G[a], (c[0], c[1], c[2]), w * lam_F[:, a])
    lam_x *= free / dg
    # G_a(c) = sum_m g_m (P(c + m e_a) - P(c - m e_a)) / dg  ->  lam_P(c +- m e_a) += +- g_m lam_G_a(c) / dg
    lam_P = np.zeros_like(Pp)
    for a in range(3):
        for m, gm in enumerate(g, start=1):
            _shift_add(lam_P, gm * lam_G[a] / dg, a, m, 1.0)
            _shift_add(lam_P, gm * lam_G[a] / dg, a, -m, -1.0)
    return lam_x, lam_P


def laplacian_on_interior_T(lam_int, dg, order=2):
    """Adjoint of ``pm.laplacian_on_interior`` (padded -> interior) at FDA order n."""
    P = order
    Ng = lam_int.shape[0]
    s = fda.second_derivative_coefficients(order)
    out = np.zeros((Ng + 2 * P,) * 3)
    c = slice(P, Ng + P)
    out[c, c, c] += 3.0 * s[0] * lam_int
    for m in range(1, len(s)):
        hi, lo = slice(P + m, Ng + P + m), slice(P - m, Ng + P - m)
        out[hi, c, c] += s[m] * lam_int
        out[lo, c, c] += s[m] * lam_int
        out[c, hi, c] += s[m] * lam_int
        out[c, lo, c] += s[m] * lam_int
        out[c, c, hi] += s[m] * lam_int
        out[c, c, lo] += s[m] * lam_int
    return out / dg**2


def box_force_vjp(xloc, dg, Ng, Nsc, phi_bc_padded, lam_F, order=2):
    """VJP of ``pm.box_force`` (F only): returns (lam_x, lam_phi_bc_padded)."""
    P = order
    delta, _ = pm.cic_deposit_box(xloc, dg, Ng, Nsc)
    phi = pm.dirichlet_potential(delta, phi_bc_padded, dg, order)
    lam_x, lam_P = interp_vjp(phi, xloc, dg, lam_F, order)
    inside = boundary.interior_mask(Ng, order)
    lam_int = lam_P[P:Ng + P, P:Ng + P, P:Ng + P]
    lam_src = pm.zero_bc_poisson(lam_int, dg, order)     # self-adjoint Dirichlet solve (S Lambda^-1 S)
    lam_bc = np.where(inside, 0.0, lam_P)                # ghost layers take Phi_BC directly
    lam_bc -= np.where(inside, 0.0, laplacian_on_interior_T(lam_src, dg, order))
    lam_x += box_density_vjp(xloc, dg, Ng, Nsc, lam_src)
    return lam_x, lam_bc


def trilinear_periodic_T(vals, L, N, X):
    """Adjoint of ``boundary.trilinear_periodic`` (grid -> points): scatter to the grid."""
    d = L / N
    u = X / d - 0.5
    i0 = np.floor(u).astype(np.int64)
    f = u - i0
    out = np.zeros((N, N, N))
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                w = ((f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1])
                     * (f[:, 2] if dz else 1 - f[:, 2]))
                np.add.at(out, ((i0[:, 0] + dx) % N, (i0[:, 1] + dy) % N, (i0[:, 2] + dz) % N), w * vals)
    return out


def bc_shell_T(lam_shell, L, N, origin, dg, Ng, order=2):
    """Adjoint of ``boundary.bc_shell`` with respect to phi1."""
    c = boundary.padded_cell_index(Ng, order).astype(np.float64)
    cx, cy, cz = np.meshgrid(c, c, c, indexing="ij")
    X = np.stack([origin[0] + (cx.ravel() + 0.5) * dg, origin[1] + (cy.ravel() + 0.5) * dg,
                  origin[2] + (cz.ravel() + 0.5) * dg], axis=1)
    vals = np.where(boundary.interior_mask(Ng, order), 0.0, lam_shell).ravel()
    return trilinear_periodic_T(vals, L, N, X)


def central_gradient_T(g, L, order=2):
    """Adjoint of ``lpt.central_gradient``: the central difference is antisymmetric."""
    N = g.shape[1]
    d = L / N
    cf = fda.gradient_coefficients(order)
    return -sum(gm * (np.roll(g[a], -m, axis=a) - np.roll(g[a], m, axis=a)) / d
                for a in range(3) for m, gm in enumerate(cf, start=1))


def lpt_vjp(delta, L, lam_phi1, lam_psi1, lam_psi2, order=2):
    """lam_delta_i from the adjoints of phi1, Psi1 and Psi2 (Eqs. 5-6, C.2)."""
    N = delta.shape[0]
    d = L / N
    lam = lpt.laplacian_symbol(N, L, order)

    def inv(fk):
        out = np.where(lam != 0, fk / np.where(lam != 0, lam, 1.0), 0.0)
        out[0, 0, 0] = 0.0                   # the k = 0 mode is removed (by index)
        return out
    kx, ky, kz = ics.fourier_wavenumbers(N, L)
    D = [fda.gradient_symbol(k, d, order) for k in (kx, ky, kz)]
    phi1_k = inv(np.fft.rfftn(delta))
    sec = lambda i, j, fk: np.fft.irfftn(-D[i] * D[j] * fk, s=delta.shape, axes=(0, 1, 2))
    xx, yy, zz = sec(0, 0, phi1_k), sec(1, 1, phi1_k), sec(2, 2, phi1_k)
    xy, xz, yz = sec(0, 1, phi1_k), sec(0, 2, phi1_k), sec(1, 2, phi1_k)
    lam_phi2 = central_gradient_T(lam_psi2, L, order)
    lam_S = np.fft.irfftn(inv(np.fft.rfftn(lam_phi2)), s=delta.shape, axes=(0, 1, 2))
    parts = [((0, 0), lam_S * (yy + zz)), ((1, 1), lam_S * (xx + zz)), ((2, 2), lam_S * (xx + yy)),
             ((0, 1), -2.0 * lam_S * xy), ((0, 2), -2.0 * lam_S * xz), ((1, 2), -2.0 * lam_S * yz)]
    lam_phi1_k = np.fft.rfftn(lam_phi1 + central_gradient_T(lam_psi1, L, order))
    for (i, j), v in parts:
        lam_phi1_k = lam_phi1_k + (-D[i] * D[j]) * np.fft.rfftn(v)
    return np.fft.irfftn(inv(lam_phi1_k), s=delta.shape, axes=(0, 1, 2))


# ----------------------------------------------------------------------------- full run
def forward_with_checkpoints(w, cfg):
    """The method's run from white noise w, keeping what the reverse sweep needs: the
    initial fields, every box's displacements at each force evaluation (checkpoints), and
    the final global positions x = (q + s) mod L and momenta p (L+, Eq. 55)."""
    order = getattr(cfg, "fda_order", 2)
    w = np.asarray(w, dtype=np.float64)
    fields = scola.initial_fields(w, cfg)
    sched = scola.schedule(cfg)
    n = len(sched["alpha"])
    Np3 = cfg.Np**3
    boxes = []
    for b in range(cfg.nboxes):
        g = scola.box_geometry(cfg, b)
        # per-tile final scale factors: the box's own KDK schedule (same a_i, same step count)
        sb = scola.box_schedule(cfg, b) if getattr(cfg, "a_final", None) is not None else sched
        ids = tiling.box_global_ids(cfg.Np, cfg.Ntiles, g.t, g.Nbuf)
        psi1 = fields.psi1.reshape(3, -1)[:, ids].T
        psi2 = fields.psi2.reshape(3, -1)[:, ids].T
        qloc = (tiling.box_local_lattice(g.Nsc) + 0.5) * (cfg.L / cfg.Np)
        shell = boundary.bc_shell(fields.phi1, cfg.L, g.origin, g.dg, g.Ng, order)
        s = -sb["D1_i"] * psi1 + sb["D2_i"] * psi2
        p = np.zeros_like(s)
        ss = []
        for k in range(n + 1):
            ss.append(s)
            F = pm.box_force(qloc + s, g.dg, g.Ng, g.Nsc, sb["D1"][k] * shell, order=order)["F"]
            D1, D2 = sb["D1"][k], sb["D2"][k]
            p = p + sb["beta"][k] * (F - D1 * psi1 + (D2 - D1 * D1) * psi2)
            if k < n:
                s = s + sb["alpha"][k] * p - sb["dD1"][k] * psi1 + sb["dD2"][k] * psi2
        a_f = scola.box_final_a(cfg, b)
        p_fin = p + scola.lpt_momentum(a_f, sb["dD1da_f"], sb["dD2da_f"], psi1, psi2, cfg)
        boxes.append(dict(sb=sb, g=g, ids=ids, psi1=psi1, psi2=psi2, qloc=qloc, shell=shell, ss=ss, s=s,
                          p=p_fin, a_f=a_f))
    s_glob = np.zeros((Np3, 3))
    p_glob = np.zeros((Np3, 3))
    for bx in boxes:
        keep = tiling.tile_interior_mask(cfg.Np, cfg.Ntiles, bx["g"].Nbuf)
        s_glob[bx["ids"][keep]] = bx["s"][keep]
        p_glob[bx["ids"][keep]] = bx["p"][keep]
    x = np.mod(scola.lattice_positions(cfg.Np, cfg.L) + s_glob, cfg.L)
    return dict(fields=fields, boxes=boxes, n=n, order=order, x=x, p=p_glob)


def final_state_vjp(state, cfg, lam_x, lam_p=None):
    """dL/dw from dL/dx and dL/dp of the final global arrays of ``forward_with_checkpoints``.

    x = (q + s) mod L (Sec. 2.1, Eq. 1) gives lam_s = lam_x for every tile particle; the
    momentum p = p_res + a_f^2 calH(a_f) (-dD1/da Psi1 + dD2/da Psi2) (L+, Eq. 55) gives
    lam_p_res = lam_p and lam_Psi1 = -c lam_p dD1/da, lam_Psi2 = c lam_p dD2/da with
    c = a_f^2 calH(a_f).  Buffer particles of a box leave no output, so they start at zero.
    Then the KDK sequence in reverse, L-, the shell, 2LPT and the colouring."""
    order, n, fields = state["order"], state["n"], state["fields"]
    Np3 = cfg.Np**3
    lam_x = np.asarray(lam_x, dtype=np.float64)
    lam_p = np.zeros((Np3, 3)) if lam_p is None else np.asarray(lam_p, dtype=np.float64)
    lam_psi1 = np.zeros((Np3, 3))
    lam_psi2 = np.zeros((Np3, 3))
    lam_phi1 = np.zeros_like(fields.phi1)
    for bx in state["boxes"]:
        g, sb = bx["g"], bx["sb"]
        keep = tiling.tile_interior_mask(cfg.Np, cfg.Ntiles, g.Nbuf)
        lam_s = np.zeros_like(bx["s"])
        lam_s[keep] = lam_x[bx["ids"][keep]]
        lam_p_res = np.zeros_like(lam_s)
        lam_p_res[keep] = lam_p[bx["ids"][keep]]
        c = bx["a_f"] ** 2 * cosmology.conformal_hubble(bx["a_f"], cfg.Om, cfg.OL)
        lp1 = -c * sb["dD1da_f"] * lam_p_res
        lp2 = c * sb["dD2da_f"] * lam_p_res
        lam_pk = lam_p_res
        lam_shell = np.zeros((g.Ng + 2 * order,) * 3)
        for k in range(n, -1, -1):
            if k < n:
                lam_pk = lam_pk + sb["alpha"][k] * lam_s
                lp1 = lp1 - sb["dD1"][k] * lam_s
                lp2 = lp2 + sb["dD2"][k] * lam_s
            b = sb["beta"][k]
            D1, D2 = sb["D1"][k], sb["D2"][k]
            lam_F = b * lam_pk
            lp1 = lp1 - b * D1 * lam_pk
            lp2 = lp2 + b * (D2 - D1 * D1) * lam_pk
            lx, lbc = box_force_vjp(bx["qloc"] + bx["ss"][k], g.dg, g.Ng, g.Nsc, D1 * bx["shell"], lam_F, order)
            lam_s = lam_s + lx
            lam_shell += D1 * lbc
        lp1 = lp1 - sb["D1_i"] * lam_s
        lp2 = lp2 + sb["D2_i"] * lam_s
        np.add.at(lam_psi1, bx["ids"], lp1)
        np.add.at(lam_psi2, bx["ids"], lp2)
        lam_phi1 += bc_shell_T(lam_shell, cfg.L, cfg.Np, g.origin, g.dg, g.Ng, order)
    N = cfg.Np
    if getattr(cfg, "lpt_order", 2) == 1:
        lam_psi2[:] = 0.0          # Zel'dovich frame: Psi2 = 0 does not depend on the noise
    lam_delta = lpt_vjp(fields.delta, cfg.L, lam_phi1, lam_psi1.T.reshape(3, N, N, N),
                        lam_psi2.T.reshape(3, N, N, N), order)
    return ics.initial_density(lam_delta, cfg.L, cfg.Om, cfg.h, cfg.ns, cfg.sigma8)


def loss_and_grad(w, cfg, delta_target):
    """Lval(w) and dLval/dw for the final-density loss of one sCOLA run: the periodic CIC
    adjoint of the final density (Sec. 4.1) gives lam_x, then ``final_state_vjp``."""
    state = forward_with_checkpoints(w, cfg)
    x = state["x"]
    delta_f = stats.cic_density_periodic(x, cfg.L, cfg.Np, cfg.Np)
    resid = delta_f - delta_target
    value = float(np.sum(resid**2))
    lam_x = periodic_density_vjp(x, cfg.L, cfg.Np, cfg.Np, 2.0 * resid)
    return value, final_state_vjp(state, cfg, lam_x)
