"""NumPy re-enactment of the GPU solve on the host-exported packed operators.

Test helper only: it replays, phase by phase and with the same packed data
the GPU kernel consumes (exported by ``bddc_host_setup_*``), the arithmetic of
the persistent kernel (Step 1, Step 2, f*, PCG with the BDDC preconditioner,
post-correction).  Comparing it with the oracle checks the native setup and
the data layout on a machine without a GPU; the GPU itself is compared with
the oracle directly in the ``-m gpu`` tests.
"""

from __future__ import annotations

import numpy as np


class Packed:
    def __init__(self, hs):
        for name in ("sub_inst", "sub_ng", "sub_ni", "sub_nc", "sub_m", "sub_local", "slot_g", "slot_partner",
                     "cslot_c", "c_slot_a", "c_slot_b", "inst_goff", "inst_ng", "inst_coff", "inst_ncn",
                     "inst_ncf", "inst_kinv_off", "inst_s0", "inst_s1", "inst_face_off", "inst_nfaces",
                     "inst_cell_off", "inst_ncells", "off_S", "off_F", "off_P", "off_Gpre", "off_Gpost",
                     "off_slot", "off_cslot", "off_cell", "off_int", "cell_gid", "int_fid", "g_fid",
                     "inst_vol", "sub_d", "slot_w", "slot_dsig", "g_bsign", "S", "F", "P", "Gpre",
                     "Gpost", "Kinv", "slot_fcs", "cslot_n", "slot_coef", "P64",
                     "slot_fk", "slot_fopp", "slot_fcell"):
            setattr(self, name, hs.get(name))
        # sparse coarse solver: no dense inverse; coarse solves go through
        # the host sweeps over the packed multifrontal factor
        self.coarse_sparse = len(hs.get("cn_p")) > 0
        self.hs = hs
        self.n_sub = len(self.sub_ng)
        self.n_inst = len(self.inst_ng)
        self.G = int(self.inst_ng.sum())

    def mat(self, arr, off, s, n_in, n_out):
        """Operator stored input-major -> dense (n_out x n_in)."""
        o = int(off[s])
        return arr[o:o + n_in * n_out].reshape(n_in, n_out).T

    def slots(self, s):
        a, b = int(self.off_slot[s]), int(self.off_slot[s + 1])
        return np.arange(a, b)


def full_form_apply(P: Packed, s, d, dp):
    """Interface rows of the full-space form of the Step-3 operator for
    subdomain s (BDDC_FORM_FULL): the direction d (local slots) and its
    pressure constant dp extended into the subdomain by the interface columns
    of G_post, then per interface face the row of its cell's RT0 mass block
    plus the cell's +-pressure, from the exported per-slot face data."""
    ng, ni, nc = int(P.sub_ng[s]), int(P.sub_ni[s]), int(P.sub_nc[s])
    sl = P.slots(s)
    G = P.mat(P.Gpost, P.off_Gpost, s, ng + nc, ni + nc)
    ext = G[:, :ng] @ d
    loc = np.concatenate([d, ext[:ni]])
    fk, fo, fc = P.slot_fk[sl], P.slot_fopp[sl], P.slot_fcell[sl]
    uo = np.where(fo >= 0, loc[np.maximum(fo, 0)], 0.0)
    pk = P.sub_d[s] * (dp + ext[ni + np.abs(fc) - 1])
    return fk * (d / 3.0 + uo / 6.0) + np.sign(fc) * pk


def emulate_solve(P: Packed, f, bc, tol, maxit=5000, mixed=False, full_form=False):
    """Returns (flux, pressure, iterations per instance, alphas, betas).

    full_form=True applies the Step-3 operator in its full-space form
    (full_form_apply) instead of S^i.

    mixed=True replays the mixed-precision kernel: F and Psi applied as
    P_Z F P_Z and Psi_0 + P_Z Psi (P_Z removes each face's net flux, Psi_0
    carries the exact unit net fluxes), and the closing FP64 coarse pressure
    correction (F and P must then hold the FP32-rounded operators)."""
    G, ns = P.G, P.n_sub
    ng, m, nc, ni = P.sub_ng, P.sub_m, P.sub_nc, P.sub_ni
    S = [P.mat(P.S, P.off_S, s, ng[s], ng[s]) for s in range(ns)]
    F = [P.mat(P.F, P.off_F, s, ng[s], ng[s]) for s in range(ns)]
    PsiT = [P.P[P.off_P[s]:P.off_P[s] + m[s] * ng[s]].reshape(m[s], ng[s]) for s in range(ns)]
    Gpre = [P.mat(P.Gpre, P.off_Gpre, s, nc[s], ng[s]) for s in range(ns)]
    Gpost = [P.mat(P.Gpost, P.off_Gpost, s, ng[s] + nc[s], ni[s] + nc[s]) for s in range(ns)]
    slots = [P.slots(s) for s in range(ns)]
    gl = [P.slot_g[sl] for sl in slots]
    w = [P.slot_w[sl] for sl in slots]
    cid = [P.cslot_c[P.off_cslot[s]:P.off_cslot[s + 1]] for s in range(ns)]
    cells = [P.cell_gid[P.off_cell[s]:P.off_cell[s + 1]] for s in range(ns)]
    ints = [P.int_fid[P.off_int[s]:P.off_int[s + 1]] for s in range(ns)]
    inst = P.sub_inst
    fcs = [P.slot_fcs[sl] for sl in slots]
    coef = [P.slot_coef[sl] for sl in slots]
    cnt = [P.cslot_n[P.off_cslot[s]:P.off_cslot[s + 1]] for s in range(ns)]

    def pz(s, v):
        """Remove each face's net flux (symmetric projection P_Z)."""
        v = v.copy()
        for a in range(m[s]):
            if cnt[s][a] == 0:
                continue
            sel = fcs[s] == a
            v[sel] -= coef[s][sel] * np.sum(coef[s][sel] * v[sel]) / cnt[s][a]
        return v

    def psi0t(s, r):
        """Psi_0^T r: the exact unit-net-flux part of the coarse basis."""
        out = np.zeros(m[s])
        for a in range(m[s]):
            if cnt[s][a]:
                sel = fcs[s] == a
                out[a] = np.sum(coef[s][sel] * r[sel]) / cnt[s][a]
        return out

    def psi0(s, wcs):
        out = np.zeros(ng[s])
        for a in range(m[s]):
            if cnt[s][a]:
                sel = fcs[s] == a
                out[sel] += coef[s][sel] * wcs[a] / cnt[s][a]
        return out

    def prolong(s, wcs):
        if not mixed:
            return PsiT[s].T @ wcs
        return psi0(s, wcs) + pz(s, PsiT[s].T @ wcs)

    def restrict(s, r):
        if not mixed:
            return PsiT[s] @ r
        return psi0t(s, r) + PsiT[s] @ pz(s, r)

    def fapply(s, r):
        if not mixed:
            return F[s] @ r
        return pz(s, F[s] @ pz(s, r))

    def assemble(parts):
        out = np.zeros(G)
        for s in range(ns):
            np.add.at(out, gl[s], parts[s])
        return out

    def coarse(rc_parts, prhs=None):
        wc = []
        for b in range(P.n_inst):
            ncn, ncf = int(P.inst_ncn[b]), int(P.inst_ncf[b])
            rhs = np.zeros(ncn)
            for s in range(P.inst_s0[b], P.inst_s1[b]):
                np.add.at(rhs, cid[s], rc_parts[s])
            if prhs is not None:
                rhs[ncf:] = prhs[P.inst_s0[b]:P.inst_s1[b]]
            if P.coarse_sparse:
                wc.append(P.hs.coarse_solve(b, rhs))
            else:
                K = P.Kinv[P.inst_kinv_off[b]:P.inst_kinv_off[b] + ncn * ncn].reshape(ncn, ncn)
                wc.append(K @ rhs)
        return wc

    g = P.g_bsign * np.where(P.g_bsign != 0, bc[P.g_fid], 0.0)
    # Step 1
    rc = [PsiT[s] @ (w[s] * g[gl[s]]) for s in range(ns)]
    prhs = np.array([P.sub_d[s] * P.inst_vol[inst[s]] * np.sum(-f[cells[s]]) for s in range(ns)])
    wc = coarse(rc, prhs)
    u0 = assemble([w[s] * prolong(s, wc[inst[s]][cid[s]]) for s in range(ns)])
    # Step 2 and f*
    fstar = g - assemble([S[s] @ u0[gl[s]] + Gpre[s] @ f[cells[s]] for s in range(ns)])
    scale = np.zeros(P.n_inst)
    for b in range(P.n_inst):
        sl = slice(P.inst_goff[b], P.inst_goff[b] + P.inst_ng[b])
        scale[b] = np.linalg.norm(g[sl]) + np.linalg.norm(g[sl] - fstar[sl])

    def precond(r):
        rl = [w[s] * r[gl[s]] for s in range(ns)]
        wc = coarse([restrict(s, rl[s]) for s in range(ns)])
        zl = [prolong(s, wc[inst[s]][cid[s]]) + fapply(s, rl[s]) for s in range(ns)]
        z = assemble([w[s] * zl[s] for s in range(ns)])
        zp = np.array([wc[inst[s]][P.inst_ncf[inst[s]] + P.sub_local[s]] for s in range(ns)])
        return z, zp

    def op(d, dp):
        if full_form:
            return assemble([full_form_apply(P, s, d[gl[s]], dp[s]) for s in range(ns)])
        return assemble([S[s] @ d[gl[s]] + P.slot_dsig[slots[s]] * dp[s] for s in range(ns)])

    # PCG per instance (instances are independent; run them jointly)
    x = np.zeros(G)
    xp = np.zeros(ns)
    r = fstar.copy()
    z, zp = precond(r)
    its = np.zeros(P.n_inst, dtype=int)
    alphas = [[] for _ in range(P.n_inst)]
    betas = [[] for _ in range(P.n_inst)]
    done = np.zeros(P.n_inst, dtype=bool)
    islc = [slice(P.inst_goff[b], P.inst_goff[b] + P.inst_ng[b]) for b in range(P.n_inst)]
    sslc = [slice(P.inst_s0[b], P.inst_s1[b]) for b in range(P.n_inst)]
    rho = np.array([r[islc[b]] @ z[islc[b]] for b in range(P.n_inst)])
    rho0 = rho.copy()
    r0 = np.array([np.linalg.norm(r[islc[b]]) for b in range(P.n_inst)])
    for b in range(P.n_inst):
        if r0[b] <= 1e-14 * scale[b] or rho[b] <= 0.0:
            done[b] = True
            if not mixed:
                xp[sslc[b]] += zp[sslc[b]]
    d, dp = z.copy(), zp.copy()
    for k in range(maxit):
        if done.all():
            break
        q = op(d, dp)
        for b in range(P.n_inst):
            if done[b]:
                continue
            sl, ss = islc[b], sslc[b]
            alpha = rho[b] / (d[sl] @ q[sl])
            alphas[b].append(alpha)
            x[sl] += alpha * d[sl]
            xp[ss] += alpha * dp[ss]
            r[sl] -= alpha * q[sl]
        z_new, zp_new = precond(r)
        for b in range(P.n_inst):
            if done[b]:
                continue
            sl, ss = islc[b], sslc[b]
            its[b] = k + 1
            rz = r[sl] @ z_new[sl]
            nr = np.linalg.norm(r[sl])
            if nr / r0[b] <= tol or nr <= 1e-14 * scale[b] or rz <= 1e-24 * rho0[b]:
                done[b] = True
                if not mixed:
                    xp[ss] += zp_new[ss]
                continue
            beta = rz / rho[b]
            betas[b].append(beta)
            rho[b] = rz
            d[sl] = z_new[sl] + beta * d[sl]
            dp[ss] = zp_new[ss] + beta * dp[ss]
    if mixed:
        # closing coarse pressure correction with the FP64 basis
        P64 = [P.P64[P.off_P[s]:P.off_P[s] + m[s] * ng[s]].reshape(m[s], ng[s]) for s in range(ns)]
        wc = coarse([P64[s] @ (w[s] * r[gl[s]]) for s in range(ns)], np.zeros(ns))
        xp += np.array([wc[inst[s]][P.inst_ncf[inst[s]] + P.sub_local[s]] for s in range(ns)])
    # post
    flux = np.zeros(int(P.inst_nfaces.sum()))
    pres = np.zeros(int(P.inst_ncells.sum()))
    u = u0 + x
    for s in range(ns):
        flux[P.g_fid[gl[s]]] = u[gl[s]]
        out = Gpost[s] @ np.concatenate([u[gl[s]], f[cells[s]]])
        flux[ints[s]] = out[:ni[s]]
        pres[cells[s]] = P.sub_d[s] * (xp[s] + out[ni[s]:])
    return flux, pres, its, alphas, betas
