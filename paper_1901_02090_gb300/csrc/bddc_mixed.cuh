// Mixed-precision phases of the persistent solve kernel (included by
// bddc_kernels.cu inside namespace bddc, after the FP64 phases).
//
// GB300 retires FP64 arithmetic at about 1/64 of the FP32 rate (~1.6 FP64
// lane operations per clock per SM), so on this path every per-dof quantity
// of the CG recurrence (x, r, d, q, z and the local slots) is an FP32 pair
// (hi, lo) -- "double-float", 48 significant bits -- updated with
// error-free FP32 transformations.  FP64 remains for the per-instance
// scalars (alpha, beta, norms), the once-per-solve Step 1/2 and
// post-processing, and the closing coarse pressure correction.  The
// subdomain correction F and the coarse basis Psi are FP32 operators applied
// as P_Z F P_Z and Psi_0 + P_Z Psi (symmetric, exactly balanced), S and the
// coarse inverse are FP32 pairs.
#pragma once

// face means of a pair vector (vh, vl): t_a = (sum_{k in a} coef_k v_k) / n_a
// for net-flux rows a, 0 for adaptive rows (lane per row)
__device__ __forceinline__ void mx_face_means(const Params& p, int64_t s, const float* vh, const float* vl,
                                              float2* t) {
    const int m = p.sub_m[s];
    const int64_t so = p.off_slot[s], co = p.off_cslot[s];
    for (int a = threadIdx.x & 31; a < m; a += 32) {
        const int na = p.cslot_n[co + a];
        float2 acc = dd_zero();
        if (na > 0) {
            const int64_t fs = so + p.cslot_fstart[co + a];
            for (int q = 0; q < na; ++q) {
                const int k = __ldg(p.slot_fperm + fs + q);
                acc = dd_add(acc, dd_sign(make_float2(vh[k], vl[k]), __ldg(p.slot_fcoefp_f + fs + q)));
            }
            acc = dd_mul(acc, __ldg(p.cslot_inv2 + co + a));
        }
        t[a] = acc;
    }
    __syncwarp();
}

// local part of Algorithm 2 for the weighted residual held in (w.xh, w.xl):
// rc = Psi_0^T r + Psi^T P_Z r, y = P_Z F P_Z r
__device__ void mx_restrict(const Params& p, int64_t s, WarpSm w) {
    const int ng = p.sub_ng[s], m = p.sub_m[s];
    const int64_t so = p.off_slot[s], co = p.off_cslot[s];
    const int l = threadIdx.x & 31;
    float2* t = V2(w.tsum);
    float2* y = V2(w.xin);
    mx_face_means(p, s, w.xh, w.xl, t);
    for (int k = l; k < ng; k += 32) {
        const float2 v = dd_sub(make_float2(w.xh[k], w.xl[k]),
                                dd_sign(t[p.slot_fcs[so + k]], __ldg(p.slot_coef_f + so + k)));
        w.xh[k] = v.x;
        w.xl[k] = v.y;
    }
    __syncwarp();
    const float* P = reinterpret_cast<const float*>(p.P) + p.off_P[s];
    const float* F = reinterpret_cast<const float*>(p.F) + p.off_F[s];
    float2* rcl = V2(p.rcl);
    for (int a = l; a < m; a += 32) {
        const float* row = P + (int64_t)a * ng;
        float a0 = 0.0f, a1 = 0.0f;
        int k = 0;
        for (; k + 8 <= ng; k += 8) {
            float A[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) A[t] = __ldg(row + k + t);
#pragma unroll
            for (int t = 0; t < 8; t += 2) {
                a0 = fmaf(A[t], w.xh[k + t], a0);
                a1 = fmaf(A[t + 1], w.xh[k + t + 1], a1);
            }
        }
        for (; k < ng; ++k) a0 = fmaf(__ldg(row + k), w.xh[k], a0);
        rcl[co + a] = dd_add(make_float2(a0 + a1, 0.0f), t[a]);
    }
    gemv_warp(F, ng, w, [&](int o, double v) { y[o] = make_float2((float)v, 0.0f); });
    __syncwarp();
    // P_Z on y (face means of y; y's low parts are zero)
    for (int a = l; a < m; a += 32) {
        const int na = p.cslot_n[co + a];
        float2 acc = dd_zero();
        if (na > 0) {
            const int64_t fs = so + p.cslot_fstart[co + a];
            for (int q = 0; q < na; ++q)
                acc = dd_add(acc, dd_sign(y[__ldg(p.slot_fperm + fs + q)], __ldg(p.slot_fcoefp_f + fs + q)));
            acc = dd_mul(acc, __ldg(p.cslot_inv2 + co + a));
        }
        t[a] = acc;
    }
    __syncwarp();
    float2* yl = V2(p.yl);
    for (int k = l; k < ng; k += 32)
        yl[so + k] = dd_sub(y[k], dd_sign(t[p.slot_fcs[so + k]], __ldg(p.slot_coef_f + so + k)));
    __syncwarp();
}

// v = Psi_0 wcs + P_Z Psi wcs for the staged coarse values (w.wcs as pairs);
// the result is left in (w.xh, w.xl)
__device__ void mx_prolong_local(const Params& p, int64_t s, WarpSm w) {
    const int ng = p.sub_ng[s], m = p.sub_m[s];
    const int64_t so = p.off_slot[s], co = p.off_cslot[s];
    const int l = threadIdx.x & 31;
    const float2* wcs = V2(w.wcs);
    float2* t = V2(w.tsum);
    const float* P = reinterpret_cast<const float*>(p.P) + p.off_P[s];
    for (int k = l; k < ng; k += 32) {
        float acc = 0.0f;
        for (int a = 0; a < m; ++a) acc = fmaf(__ldg(P + (int64_t)a * ng + k), wcs[a].x, acc);
        w.xh[k] = acc;
        w.xl[k] = 0.0f;
    }
    __syncwarp();
    mx_face_means(p, s, w.xh, w.xl, t);
    // per row: u_a = wcs_a / n_a - mean_a
    for (int a = l; a < m; a += 32)
        if (p.cslot_n[co + a] > 0) t[a] = dd_sub(dd_mul(wcs[a], __ldg(p.cslot_inv2 + co + a)), t[a]);
    __syncwarp();
    for (int k = l; k < ng; k += 32) {
        const float2 v = dd_add(make_float2(w.xh[k], w.xl[k]),
                                dd_sign(t[p.slot_fcs[so + k]], __ldg(p.slot_coef_f + so + k)));
        w.xh[k] = v.x;
        w.xl[k] = v.y;
    }
    __syncwarp();
}

__device__ __forceinline__ void mx_stage_wc(const Params& p, int64_t s, const float2* wc_b, WarpSm w) {
    const int m = p.sub_m[s];
    const int64_t co = p.off_cslot[s];
    float2* wcs = V2(w.wcs);
    for (int a = threadIdx.x & 31; a < m; a += 32) wcs[a] = __ldcg(wc_b + p.cslot_c[co + a]);
    __syncwarp();
}

// ---- phases ------------------------------------------------------------------------------
__device__ void mx_step1(const Params& p, int64_t s, WarpSm w) {
    const int b = p.sub_inst[s];
    const int ng = p.sub_ng[s], m = p.sub_m[s], nc = p.sub_nc[s];
    const int64_t so = p.off_slot[s], co = p.off_cslot[s];
    const int l = threadIdx.x & 31;
    for (int k = l; k < ng; k += 32) {
        const int gi = p.slot_g[so + k];
        const double sg = p.g_bsign[gi];
        const double gv = sg != 0.0 ? sg * p.bc_in[p.g_fid[gi]] : 0.0;
        if (slot_owner((int)(so + k), p.slot_partner[so + k])) p.g[gi] = gv;
        w.x[k] = p.slot_w[so + k] * gv;
    }
    __syncwarp();
    const double* P64 = p.P64 + p.off_P[s];
    float2* rcl = V2(p.rcl);
    for (int a = l; a < m; a += 32) {
        double acc = 0.0;
        for (int k = 0; k < ng; ++k) acc = fma(__ldg(P64 + (int64_t)a * ng + k), w.x[k], acc);
        rcl[co + a] = dd_of(acc);
    }
    double v = 0.0;
    const int64_t cb = p.off_cell[s];
    for (int r = l; r < nc; r += 32) v += -p.f_in[p.cell_gid[cb + r]];
    v = warp_sum(v);
    if (l == 0) p.prhs[s] = p.sub_d[s] * p.inst_vol[b] * v;
    __syncwarp();
}

// coarse solve rows (CTA per unit) in FP32-pair arithmetic: wc = Kinv * rhs
__device__ void mx_coarse(const Params& p, int64_t u, bool step1, double* rhs_area, int& staged) {
    const int b = p.cunit_inst[u];
    if (!step1 && inst_done_block(p, b)) return;
    const int64_t ncn = p.inst_ncn[b], ncf = p.inst_ncf[b], coff = p.inst_coff[b];
    const int64_t cfo = p.inst_cfoff[b];
    const int64_t ncols = step1 ? ncn : ncf;
    float2* rhs = V2(rhs_area);
    const float2* rcl = V2(p.rcl);
    if (staged != b) {
        __syncthreads();
        const int64_t s0 = p.inst_s0[b];
        for (int64_t c = threadIdx.x; c < ncols; c += kThreads) {
            float2 v;
            if (c < ncf) {
                const int a = p.c_slot_a[cfo + c], bb = p.c_slot_b[cfo + c];
                v = a >= 0 ? __ldcg(rcl + a) : dd_zero();
                if (bb >= 0) v = dd_add(v, __ldcg(rcl + bb));
            } else {
                v = dd_of(__ldcg(p.prhs + s0 + (c - ncf)));
            }
            rhs[c] = v;
        }
        __syncthreads();
        staged = b;
    }
    const float2* K = reinterpret_cast<const float2*>(p.Kinv) + p.inst_kinv_off[b];
    const uint64_t pol = l2_stream_policy();
    const int wi = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int64_t r0 = p.cunit_row0[u];
    const int64_t r1 = (r0 + p.coarse_rows < ncn) ? r0 + p.coarse_rows : ncn;
    float2* wc = V2(p.wc);
    for (int64_t row = r0 + wi; row < r1; row += kWarps) {
        const float2* kr = K + row * ncn;
        float sh = 0.0f, sl = 0.0f;
        int64_t c = l;
        for (; c + 7 * 32 < ncols; c += 8 * 32) {
            float2 A[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) A[t] = ld_hint(kr + c + 32 * t, pol);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const float2 xv = rhs[c + 32 * t];
                dd_acc(sh, sl, A[t], xv.x, xv.y);
            }
        }
        for (; c < ncols; c += 32) {
            const float2 xv = rhs[c];
            dd_acc(sh, sl, ld_hint(kr + c, pol), xv.x, xv.y);
        }
        const float2 acc = dd_warp_sum(dd_quick(sh, sl));
        if (l == 0) wc[coff + row] = acc;
    }
}

__device__ void mx_u0(const Params& p, int64_t s, WarpSm w) {
    const int b = p.sub_inst[s];
    const int ng = p.sub_ng[s];
    const int64_t so = p.off_slot[s];
    mx_stage_wc(p, s, V2(p.wc) + p.inst_coff[b], w);
    mx_prolong_local(p, s, w);
    for (int k = threadIdx.x & 31; k < ng; k += 32)
        p.tl[so + k] = p.slot_w[so + k] * dd_dbl(make_float2(w.xh[k], w.xl[k]));
    __syncwarp();
}

// f* (FP64, once per solve), r_0 = f* and x_0 = 0 as pairs, then restrict r_0
__device__ void mx_fstar(const Params& p, int64_t s, WarpSm w) {
    const int ng = p.sub_ng[s];
    const int64_t so = p.off_slot[s];
    const int l = threadIdx.x & 31;
    float2* r0 = V2(p.rbuf0);
    float2* x = V2(p.x);
    float2* rl = V2(p.rl);
    double rr = 0.0, a1 = 0.0, a2 = 0.0;
    for (int k = l; k < ng; k += 32) {
        const int pt = p.slot_partner[so + k];
        const int gi = p.slot_g[so + k];
        const double gv = __ldcg(p.g + gi);
        const double loc = __ldcg(p.ql + so + k) + (pt >= 0 ? __ldcg(p.ql + pt) : 0.0);
        const double fs = gv - loc;
        if (slot_owner((int)(so + k), pt)) {
            r0[gi] = dd_of(fs);
            x[gi] = dd_zero();
            rr += fs * fs;
            a1 += gv * gv;
            a2 += loc * loc;
        }
        const float2 wr = dd_of(p.slot_w[so + k] * fs);
        w.xh[k] = wr.x;
        w.xl[k] = wr.y;
        rl[so + k] = wr;
    }
    rr = warp_sum(rr);
    a1 = warp_sum(a1);
    a2 = warp_sum(a2);
    if (l == 0) {
        p.part_rr[s] = rr;
        p.part_a1[s] = a1;
        p.part_a2[s] = a2;
        p.xp[s] = 0.0;
        p.dp0[s] = 0.0;
        p.dp1[s] = 0.0;
    }
    __syncwarp();
    publish_total(p, p.sub_inst[s], 1, kCtrRR, 0, true);
    mx_restrict(p, s, w);
}

__device__ bool mx_prolong(const Params& p, int64_t s, WarpSm w) {
    const int b = p.sub_inst[s];
    if (inst_done(p, b)) return false;
    const int ng = p.sub_ng[s];
    const int64_t so = p.off_slot[s];
    const float2* wcb = V2(p.wc) + p.inst_coff[b];
    mx_stage_wc(p, s, wcb, w);
    mx_prolong_local(p, s, w);
    const float2* yl = V2(p.yl);
    const float2* rl = V2(p.rl);
    float2* zl = V2(p.zl);
    float2 rz = dd_zero();
    for (int k = threadIdx.x & 31; k < ng; k += 32) {
        const float2 z = dd_add(make_float2(w.xh[k], w.xl[k]), __ldcg(yl + so + k));
        zl[so + k] = dd_mul(__ldg(p.slot_w2 + so + k), z);
        rz = dd_add(rz, dd_mul(__ldcg(rl + so + k), z));
    }
    rz = dd_warp_sum(rz);
    if ((threadIdx.x & 31) == 0) {
        p.part_rz[s] = dd_dbl(rz);
        p.zp[s] = dd_dbl(__ldcg(wcb + p.inst_ncf[b] + p.sub_local[s]));
    }
    __syncwarp();
    return true;
}

// direction update and operator apply (pairs), for the outputs [ob, oe) of
// operator-apply unit u of subdomain s (the unit with ob = 0 also stores
// the subdomain's new direction)
__device__ bool mx_dirop(const Params& p, int64_t u, int64_t s, int ob, int oe, int k, WarpSm w) {
    const int b = p.sub_inst[s];
    if (inst_done(p, b)) return false;
    const int l = threadIdx.x & 31;
    const double beta = __ldcg(p.beta_hist + (int64_t)b * (p.maxit + 1) + k);
    const float2 beta2 = dd_of(beta);
    const float2* dold = V2((k & 1) ? p.dbuf0 : p.dbuf1);
    float2* dnew = V2((k & 1) ? p.dbuf1 : p.dbuf0);
    double* dpold = (k & 1) ? p.dp0 : p.dp1;
    double* dpnew = (k & 1) ? p.dp1 : p.dp0;
    const float2* zl = V2(p.zl);
    const int ng = p.sub_ng[s];
    const int64_t so = p.off_slot[s];
    for (int kk = l; kk < ng; kk += 32) {
        const int pt = p.slot_partner[so + kk];
        const int gi = p.slot_g[so + kk];
        float2 z = __ldcg(zl + so + kk);
        if (pt >= 0) z = dd_add(z, __ldcg(zl + pt));
        const float2 dn = (k == 0) ? z : dd_add(z, dd_mul(beta2, __ldcg(dold + gi)));
        if (ob == 0 && slot_owner((int)(so + kk), pt)) dnew[gi] = dn;
        w.xh[kk] = dn.x;
        w.xl[kk] = dn.y;
    }
    const double dpn = (k == 0) ? __ldcg(p.zp + s) : __ldcg(p.zp + s) + beta * __ldcg(dpold + s);
    if (l == 0 && ob == 0) dpnew[s] = dpn;
    const float2 dpn2 = dd_of(dpn);
    __syncwarp();
    const float2* S = reinterpret_cast<const float2*>(p.S) + p.off_S[s];
    float2* ql = V2(p.ql);
    float2 dq = dd_zero();
    gemv_warp_range(S, ng, ob, oe, w, [&](int kk, float2 y) {
        const float2 q = dd_add(y, dd_mul(__ldg(p.slot_dsig2 + so + kk), dpn2));
        ql[so + kk] = q;
        dq = dd_add(dq, dd_mul(make_float2(w.xh[kk], w.xl[kk]), q));
    });
    dq = dd_warp_sum(dq);
    if (l == 0) p.part_dq[u] = dd_dbl(dq);
    __syncwarp();
    return true;
}

__device__ bool mx_update(const Params& p, int64_t s, int k, WarpSm w) {
    const int b = p.sub_inst[s];
    if (inst_done(p, b)) return false;
    const int l = threadIdx.x & 31;
    const double alpha = __ldcg(p.alpha_hist + (int64_t)b * (p.maxit + 1) + k);
    const float2 alpha2 = dd_of(alpha);
    const float2* rold = V2((k & 1) ? p.rbuf1 : p.rbuf0);
    float2* rnew = V2((k & 1) ? p.rbuf0 : p.rbuf1);
    const float2* dcur = V2((k & 1) ? p.dbuf1 : p.dbuf0);
    const double* dpcur = (k & 1) ? p.dp1 : p.dp0;
    const float2* ql = V2(p.ql);
    float2* x = V2(p.x);
    float2* rl = V2(p.rl);
    const int ng = p.sub_ng[s];
    const int64_t so = p.off_slot[s];
    float2 rr = dd_zero();
    for (int kk = l; kk < ng; kk += 32) {
        const int pt = p.slot_partner[so + kk];
        const int gi = p.slot_g[so + kk];
        float2 q = __ldcg(ql + so + kk);
        if (pt >= 0) q = dd_add(q, __ldcg(ql + pt));
        const float2 rn = dd_sub(__ldcg(rold + gi), dd_mul(alpha2, q));
        if (slot_owner((int)(so + kk), pt)) {
            rnew[gi] = rn;
            x[gi] = dd_add(__ldcg(x + gi), dd_mul(alpha2, __ldcg(dcur + gi)));
            rr = dd_add(rr, dd_mul(rn, rn));
        }
        const float2 wr = dd_mul(__ldg(p.slot_w2 + so + kk), rn);
        w.xh[kk] = wr.x;
        w.xl[kk] = wr.y;
        rl[so + kk] = wr;
    }
    rr = dd_warp_sum(rr);
    if (l == 0) {
        p.part_rr[s] = dd_dbl(rr);
        p.xp[s] = __ldcg(p.xp + s) + alpha * __ldcg(dpcur + s);
    }
    __syncwarp();
    mx_restrict(p, s, w);
    return true;
}

// closing FP64 coarse pressure correction: FP64 restriction of the final
// residual (stored as pairs), coarse solve, x_p += p_0
__device__ void mx_final_restrict(const Params& p, int64_t s, WarpSm w) {
    const int b = p.sub_inst[s];
    const int ng = p.sub_ng[s], m = p.sub_m[s];
    const int64_t so = p.off_slot[s], co = p.off_cslot[s];
    const int it = __ldcg(&p.st[b].iterations);
    const float2* r = V2((it & 1) ? p.rbuf1 : p.rbuf0);
    for (int k = threadIdx.x & 31; k < ng; k += 32)
        w.x[k] = p.slot_w[so + k] * dd_dbl(__ldcg(r + p.slot_g[so + k]));
    __syncwarp();
    const double* P64 = p.P64 + p.off_P[s];
    float2* rcl = V2(p.rcl);
    for (int a = threadIdx.x & 31; a < m; a += 32) {
        double acc = 0.0;
        for (int k = 0; k < ng; ++k) acc = fma(__ldg(P64 + (int64_t)a * ng + k), w.x[k], acc);
        rcl[co + a] = dd_of(acc);
    }
    __syncwarp();
}

__device__ void mx_final_pressure(const Params& p, int64_t s) {
    if ((threadIdx.x & 31) != 0) return;
    const int b = p.sub_inst[s];
    const float2* wcb = V2(p.wc) + p.inst_coff[b];
    p.xp[s] = __ldcg(p.xp + s) + dd_dbl(__ldcg(wcb + p.inst_ncf[b] + p.sub_local[s]));
}

__device__ void mx_post(const Params& p, int64_t s, WarpSm w) {
    const int ng = p.sub_ng[s], ni = p.sub_ni[s], nc = p.sub_nc[s];
    const int64_t so = p.off_slot[s], cb = p.off_cell[s], ib = p.off_int[s];
    const int l = threadIdx.x & 31;
    const float2* x = V2(p.x);
    for (int k = l; k < ng; k += 32) {
        const int gi = p.slot_g[so + k];
        const double u = __ldcg(p.u0 + gi) + dd_dbl(__ldcg(x + gi));
        if (slot_owner((int)(so + k), p.slot_partner[so + k])) p.flux_out[p.g_fid[gi]] = u;
        w.xin[k] = u;
    }
    int nz = 0;
    for (int r = l; r < nc; r += 32) {
        const double fv = p.f_in[p.cell_gid[cb + r]];
        w.xin[ng + r] = fv;
        nz |= (fv != 0.0);
    }
    // a subdomain without sources has f = 0: its f columns contribute exactly nothing
    const int nin = ng + (__any_sync(0xffffffffu, nz) ? nc : 0);
    __syncwarp();
    float2* xin2 = V2(w.xin);  // the inputs as FP32 pairs, in place
    for (int k = l; k < nin; k += 32) xin2[k] = dd_of(w.xin[k]);
    __syncwarp();
    const float2* G = p.Gpost2 + p.off_Gpost[s];
    const int no = ni + nc;
    const double d = p.sub_d[s];
    const double xp = __ldcg(p.xp + s);
    for (int o = l; o < no; o += 32) {
        float h = 0.0f, lo = 0.0f;
        int j = 0;
        for (; j + 8 <= nin; j += 8) {
            float2 A[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) A[t] = __ldg(G + (int64_t)(j + t) * no + o);
#pragma unroll
            for (int t = 0; t < 8; ++t) dd_acc(h, lo, A[t], xin2[j + t].x, xin2[j + t].y);
        }
        for (; j < nin; ++j) dd_acc(h, lo, __ldg(G + (int64_t)j * no + o), xin2[j].x, xin2[j].y);
        const double v = dd_dbl(dd_quick(h, lo));
        if (o < ni) p.flux_out[p.int_fid[ib + o]] = v;
        else p.p_out[p.cell_gid[cb + o - ni]] = d * (xp + v);
    }
    __syncwarp();
}
