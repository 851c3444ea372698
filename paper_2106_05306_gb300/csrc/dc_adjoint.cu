// Adjoint kernels of libdc (FP64, sm_103a): the linearisation of one converged
// time step, transposed (Sec. 4, Eq. adjoint_v and ppr_adjoint).
//
// The adjoint system of a step is
//     H z + B eta = g,    C^T z = 0,     g = dL/dv_{n+1} + h dL/dx_{n+1},
// with H = M + h^2 grad^2 W(x_{n+1}) - Delta R = P - Delta P - Delta R,
// grad^2 W_i = w_i A_i^T (I - dp_i*/d(A_i x)) A_i, and per contact node:
//   stick:    z_j = 0                      (B_j = C_j = I)
//   slip:     (n - mu t).z_j = 0           (B_j = n, C_j = n - mu t; oblique)
//             and Delta R_j = -h mu f_N b b^T / |u_T|, b = n x t
//   take-off: no constraint.
// It is solved with flexible GMRES on w -> Pi_B H K(w), where Pi_B removes the
// B components and K is a two-level preconditioner: a per-node constrained
// block inverse of H, the prefactorised P^-1 projected onto C^T z = 0, and the
// block inverse again.  Every H application is matrix-free: a per-element pass
// (the polar-factor derivative for stretch, the sphere-projection derivative
// for bending) and a fixed-order per-node gather.
#include "dc_internal.h"
#include "dc_adjoint.h"
#include "dc_obstacle.cuh"
#include "dc_polar.cuh"

namespace {

__device__ __forceinline__ d4 ld(const d4* p) {
    const double2* q = reinterpret_cast<const double2*>(p);
    double2 a = q[0], b = q[1];
    d4 r;
    r.x = a.x; r.y = a.y; r.z = b.x; r.w = b.y;
    return r;
}
__device__ __forceinline__ void st(d4* p, double x, double y, double z, double w = 0.0) {
    double2* q = reinterpret_cast<double2*>(p);
    q[0] = make_double2(x, y);
    q[1] = make_double2(z, w);
}
inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

// ----------------------------------------------------------------- per-step setup

// Per triangle at x_{n+1}: R (polar factor), S^-1, 1/tr S (reading R1).
__global__ void k_adj_setup_tri(DevMesh dm, const d4* __restrict__ x1, d4* __restrict__ tr0,
                                d4* __restrict__ tr1, d4* __restrict__ tr2, d4* __restrict__ tav) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= dm.T) return;
    int4 tr = dm.tri[t];
    d4 g = ld(dm.G + t);
    d4 a = ld(x1 + tr.x), b = ld(x1 + tr.y), c = ld(x1 + tr.z);
    double e1[3] = {b.x - a.x, b.y - a.y, b.z - a.z};
    double e2[3] = {c.x - a.x, c.y - a.y, c.z - a.z};
    double F[6];
    for (int k = 0; k < 3; ++k) {
        F[k] = e1[k] * g.x + e2[k] * g.z;
        F[3 + k] = e1[k] * g.y + e2[k] * g.w;
    }
    // R, S^-1 and 1/tr S; a collapsed triangle gets S^-1 = 0 and 1/tr S = 0, so
    // its polar derivative vanishes (reading R1)
    double R[6], sinv[3], it;
    dc_polar3x2(F, R, sinv, &it);
    const double s00 = sinv[0], s01 = sinv[1], s11 = sinv[2];
    // per vertex v of the triangle: a_v = (g_v0 R1 - g_v1 R0) / tr S, and the
    // projector P = I - R0 R0^T - R1 R1^T (the front assembly reads them for
    // every pair of the triangle's vertices instead of forming them again)
    for (int v = 0; v < 3; ++v) {
        double gv0, gv1;
        if (v == 1) { gv0 = g.x; gv1 = g.y; }
        else if (v == 2) { gv0 = g.z; gv1 = g.w; }
        else { gv0 = -(g.x + g.z); gv1 = -(g.y + g.w); }
        st(tav + 4 * (long)t + v, (gv0 * R[3] - gv1 * R[0]) * it, (gv0 * R[4] - gv1 * R[1]) * it,
           (gv0 * R[5] - gv1 * R[2]) * it);
    }
    double P[9];
    for (int r = 0; r < 3; ++r)
        for (int c2 = 0; c2 < 3; ++c2) P[3 * r + c2] = ((r == c2) ? 1.0 : 0.0) - R[r] * R[c2] - R[3 + r] * R[3 + c2];
    st(tav + 4 * (long)t + 3, P[0], P[1], P[2], P[4]);
    st(tr0 + t, R[0], R[1], R[2], s00);
    st(tr1 + t, R[3], R[4], R[5], s01);
    st(tr2 + t, s11, it, P[5], P[8]);   // tr S = t, so 1/tr S = it
}

// Per vertex at x_{n+1}: sphere-projection derivative data (q_hat, kappa = s/|q|)
// (reading R2); kappa = 0 where the projection is constant.
__global__ void k_adj_setup_bend(DevMesh dm, const d4* __restrict__ x1, d4* __restrict__ bq) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= dm.m) return;
    double q[3] = {0, 0, 0};
    for (int k = dm.bptr[b]; k < dm.bptr[b + 1]; ++k) {
        d4 x = ld(x1 + dm.bidx[k]);
        double l = dm.bval[k];
        q[0] += l * x.x; q[1] += l * x.y; q[2] += l * x.z;
    }
    double s = dm.sb[b];
    double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    if (s > 0.0 && nq > 1e-14 * s)
        st(bq + b, q[0] / nq, q[1] / nq, q[2] / nq, s / nq);
    else
        st(bq + b, 0.0, 0.0, 0.0, 0.0);
}

__device__ __forceinline__ void sym_add(double H[6], double a, const double u[3]) {
    // H += a u u^T, packed (00, 01, 02, 11, 12, 22)
    H[0] += a * u[0] * u[0]; H[1] += a * u[0] * u[1]; H[2] += a * u[0] * u[2];
    H[3] += a * u[1] * u[1]; H[4] += a * u[1] * u[2]; H[5] += a * u[2] * u[2];
}

__device__ void inv3(const double A[9], double X[9]) {
    double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    double id = 1.0 / det;
    X[0] = c00 * id; X[1] = (A[2] * A[7] - A[1] * A[8]) * id; X[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    X[3] = c01 * id; X[4] = (A[0] * A[8] - A[2] * A[6]) * id; X[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    X[6] = c02 * id; X[7] = (A[1] * A[6] - A[0] * A[7]) * id; X[8] = (A[0] * A[4] - A[1] * A[3]) * id;
}

// Per free node: the node type, slip data and the constrained inverse
// D+_j = Q (R^T H_jj Q)^-1 R^T of the diagonal block of H.
__global__ void k_adj_setup_node(DevMesh dm, AdjDev ad, const d4* __restrict__ v1) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= dm.m_free) return;
    const double h2 = ad.h * ad.h;
    double H[6] = {0, 0, 0, 0, 0, 0};
    for (int k = dm.iptr[j]; k < dm.iptr[j + 1]; ++k) {
        int e = dm.iidx[k];
        int t = e / 3, a = e - 3 * t;
        d4 g = ld(dm.G + t);
        double ga0, ga1;
        if (a == 1) { ga0 = g.x; ga1 = g.y; }
        else if (a == 2) { ga0 = g.z; ga1 = g.w; }
        else { ga0 = -(g.x + g.z); ga1 = -(g.y + g.w); }
        d4 A0 = ld(ad.tr0 + t), A1 = ld(ad.tr1 + t), A2 = ld(ad.tr2 + t);
        double R0[3] = {A0.x, A0.y, A0.z}, R1[3] = {A1.x, A1.y, A1.z};
        double s00 = A0.w, s01 = A1.w, s11 = A2.x, itr = A2.y;
        double w = h2 * dm.wt[t];
        double gg = ga0 * ga0 + ga1 * ga1;
        double gam = ga0 * ga0 * s00 + 2.0 * ga0 * ga1 * s01 + ga1 * ga1 * s11;
        double av[3] = {(ga0 * R1[0] - ga1 * R0[0]) * itr, (ga0 * R1[1] - ga1 * R0[1]) * itr,
                        (ga0 * R1[2] - ga1 * R0[2]) * itr};
        // block = w (|g|^2 I - trS a a^T - gam (I - R0 R0^T - R1 R1^T))
        double d = w * (gg - gam);
        H[0] += d; H[3] += d; H[5] += d;
        if (itr > 0.0) sym_add(H, -w / itr, av);   // no rotation term for a collapsed triangle
        sym_add(H, w * gam, R0);
        sym_add(H, w * gam, R1);
    }
    for (int k = dm.tbptr[j]; k < dm.tbptr[j + 1]; ++k) {
        int b = dm.tbidx[k];
        double l = dm.tbval[k];
        d4 q = ld(ad.bq + b);
        double w = h2 * dm.wb[b] * l * l;
        double d = w * (1.0 - q.w);
        H[0] += d; H[3] += d; H[5] += d;
        double qh[3] = {q.x, q.y, q.z};
        sym_add(H, w * q.w, qh);
    }
    double mj = dm.mass[j];
    H[0] += mj; H[3] += mj; H[5] += mj;
    int type = 0;
    int cs = ad.contact[j] >= 0 ? ad.case_[j] : 0;
    double Hf[9] = {H[0], H[1], H[2], H[1], H[3], H[4], H[2], H[4], H[5]};
    double D[9];
    if (cs == 1) {
        type = 1;
        for (int q = 0; q < 9; ++q) D[q] = 0.0;
        st(ad.slip + j, 0, 0, 0, 0);
    } else if (cs == 2) {
        type = 2;
        d4 nb = ld(ad.nb + j), f = ld(ad.f + j), v = ld(v1 + j);
        double n[3] = {nb.x, nb.y, nb.z};
        double vn = n[0] * v.x + n[1] * v.y + n[2] * v.z;
        double uT[3] = {v.x - vn * n[0], v.y - vn * n[1], v.z - vn * n[2]};
        double nt = sqrt(uT[0] * uT[0] + uT[1] * uT[1] + uT[2] * uT[2]);
        double th[3] = {uT[0] / nt, uT[1] / nt, uT[2] / nt};
        double bh[3] = {n[1] * th[2] - n[2] * th[1], n[2] * th[0] - n[0] * th[2], n[0] * th[1] - n[1] * th[0]};
        double fN = f.x * n[0] + f.y * n[1] + f.z * n[2];
        double ks = ad.h * ad.mu[j] * fN / nt;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) Hf[3 * r + c] += ks * bh[r] * bh[c];
        st(ad.slip + j, th[0], th[1], th[2], ks);
        // Q = [b, t + mu n] spans null(C^T); R = [t, b] spans null(B^T)
        double Q[3][2], Rm[3][2];
        for (int r = 0; r < 3; ++r) {
            Q[r][0] = bh[r]; Q[r][1] = th[r] + ad.mu[j] * n[r];
            Rm[r][0] = th[r]; Rm[r][1] = bh[r];
        }
        double Rt_H_Q[2][2];
        for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q) {
                double s = 0;
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c) s += Rm[r][p] * Hf[3 * r + c] * Q[c][q];
                Rt_H_Q[p][q] = s;
            }
        double det = Rt_H_Q[0][0] * Rt_H_Q[1][1] - Rt_H_Q[0][1] * Rt_H_Q[1][0];
        double iv[2][2] = {{Rt_H_Q[1][1] / det, -Rt_H_Q[0][1] / det}, {-Rt_H_Q[1][0] / det, Rt_H_Q[0][0] / det}};
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double s = 0;
                for (int p = 0; p < 2; ++p)
                    for (int q = 0; q < 2; ++q) s += Q[r][p] * iv[p][q] * Rm[c][q];
                D[3 * r + c] = s;
            }
    } else {
        inv3(Hf, D);
        st(ad.slip + j, 0, 0, 0, 0);
    }
    ad.type[j] = type;
    st(ad.dinv + 3 * j, D[0], D[1], D[2]);
    st(ad.dinv + 3 * j + 1, D[3], D[4], D[5]);
    st(ad.dinv + 3 * j + 2, D[6], D[7], D[8]);
}

// ----------------------------------------------------------------- H application

// Element pass: per triangle E = h^2 w (dF - Dp[dF]) with dF = A_t z, stored as the
// vertex-1 and vertex-2 columns E g_a^T; per vertex u = h^2 w_b (dq - Dp_b[dq]).
__global__ void k_adj_elem(DevMesh dm, AdjDev ad, const d4* __restrict__ z, d4* __restrict__ c1,
                           d4* __restrict__ c2, d4* __restrict__ bu) {
    int id = blockIdx.x * blockDim.x + threadIdx.x;
    const double h2 = ad.h * ad.h;
    if (id < dm.T) {
        int4 tr = dm.tri[id];
        if (ad.mask && ad.mask[ad.node_inst[tr.x]] == 0.0) return;
        d4 g = ld(dm.G + id);
        d4 z0 = ld(z + tr.x), z1 = ld(z + tr.y), z2 = ld(z + tr.z);
        double e1[3] = {z1.x - z0.x, z1.y - z0.y, z1.z - z0.z};
        double e2[3] = {z2.x - z0.x, z2.y - z0.y, z2.z - z0.z};
        double dF0[3], dF1[3];
        for (int k = 0; k < 3; ++k) {
            dF0[k] = e1[k] * g.x + e2[k] * g.z;
            dF1[k] = e1[k] * g.y + e2[k] * g.w;
        }
        d4 A0 = ld(ad.tr0 + id), A1 = ld(ad.tr1 + id), A2 = ld(ad.tr2 + id);
        double R0[3] = {A0.x, A0.y, A0.z}, R1[3] = {A1.x, A1.y, A1.z};
        double s00 = A0.w, s01 = A1.w, s11 = A2.x, itr = A2.y;
        double r00 = R0[0] * dF0[0] + R0[1] * dF0[1] + R0[2] * dF0[2];
        double r01 = R0[0] * dF1[0] + R0[1] * dF1[1] + R0[2] * dF1[2];
        double r10 = R1[0] * dF0[0] + R1[1] * dF0[1] + R1[2] * dF0[2];
        double r11 = R1[0] * dF1[0] + R1[1] * dF1[1] + R1[2] * dF1[2];
        double om = (r10 - r01) * itr;
        double w = h2 * dm.wt[id];
        double E0[3], E1[3];
        for (int k = 0; k < 3; ++k) {
            double p0 = dF0[k] - R0[k] * r00 - R1[k] * r10;   // (I - R R^T) dF, column 0
            double p1 = dF1[k] - R0[k] * r01 - R1[k] * r11;   // column 1
            double dR0 = om * R1[k] + p0 * s00 + p1 * s01;    // R Om + (..) S^-1, column 0
            double dR1 = -om * R0[k] + p0 * s01 + p1 * s11;   // column 1
            E0[k] = w * (dF0[k] - dR0);
            E1[k] = w * (dF1[k] - dR1);
        }
        st(c1 + id, E0[0] * g.x + E1[0] * g.y, E0[1] * g.x + E1[1] * g.y, E0[2] * g.x + E1[2] * g.y);
        st(c2 + id, E0[0] * g.z + E1[0] * g.w, E0[1] * g.z + E1[1] * g.w, E0[2] * g.z + E1[2] * g.w);
        return;
    }
    int b = id - dm.T;
    if (b >= dm.m) return;
    if (ad.mask && ad.mask[ad.node_inst[b]] == 0.0) return;
    double dq[3] = {0, 0, 0};
    for (int k = dm.bptr[b]; k < dm.bptr[b + 1]; ++k) {
        d4 zz = ld(z + dm.bidx[k]);
        double l = dm.bval[k];
        dq[0] += l * zz.x; dq[1] += l * zz.y; dq[2] += l * zz.z;
    }
    d4 q = ld(ad.bq + b);
    double qd = q.x * dq[0] + q.y * dq[1] + q.z * dq[2];
    double w = h2 * dm.wb[b];
    double k1 = 1.0 - q.w;
    st(bu + b, w * (k1 * dq[0] + q.w * qd * q.x), w * (k1 * dq[1] + q.w * qd * q.y),
       w * (k1 * dq[2] + q.w * qd * q.z));
}

// Gather of the element pass.  mode 0: out = Pi_B (H z)  (free nodes)
//                               mode 1: out = w - Pi_B (H z)
//                               mode 2: out = w - H z (no projection; free nodes)
//                               mode 3: out = element part only (all m nodes)
__global__ void k_adj_gather(DevMesh dm, AdjDev ad, int mode, const d4* __restrict__ z,
                             const d4* __restrict__ c1, const d4* __restrict__ c2,
                             const d4* __restrict__ bu, const d4* __restrict__ w, d4* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int n = (mode == 3) ? dm.m : dm.m_free;
    if (i >= n) return;
    if (ad.mask && ad.mask[ad.node_inst[i]] == 0.0) return;
    double r0 = 0, r1 = 0, r2 = 0;
    for (int k = dm.iptr[i]; k < dm.iptr[i + 1]; ++k) {
        int e = dm.iidx[k];
        int t = e / 3, a = e - 3 * t;
        if (a == 1) {
            d4 c = ld(c1 + t);
            r0 += c.x; r1 += c.y; r2 += c.z;
        } else if (a == 2) {
            d4 c = ld(c2 + t);
            r0 += c.x; r1 += c.y; r2 += c.z;
        } else {
            d4 ca = ld(c1 + t), cb = ld(c2 + t);
            r0 -= ca.x + cb.x; r1 -= ca.y + cb.y; r2 -= ca.z + cb.z;
        }
    }
    for (int k = dm.tbptr[i]; k < dm.tbptr[i + 1]; ++k) {
        double l = dm.tbval[k];
        d4 u = ld(bu + dm.tbidx[k]);
        r0 += l * u.x; r1 += l * u.y; r2 += l * u.z;
    }
    if (mode == 3) {
        st(out + i, r0, r1, r2);
        return;
    }
    d4 zi = ld(z + i);
    double mi = dm.mass[i];
    r0 += mi * zi.x; r1 += mi * zi.y; r2 += mi * zi.z;
    int type = ad.type[i];
    if (type == 2) {
        d4 sl = ld(ad.slip + i);
        d4 nb = ld(ad.nb + i);
        double th[3] = {sl.x, sl.y, sl.z};
        double n[3] = {nb.x, nb.y, nb.z};
        double bh[3] = {n[1] * th[2] - n[2] * th[1], n[2] * th[0] - n[0] * th[2], n[0] * th[1] - n[1] * th[0]};
        double bz = sl.w * (bh[0] * zi.x + bh[1] * zi.y + bh[2] * zi.z);
        r0 += bz * bh[0]; r1 += bz * bh[1]; r2 += bz * bh[2];
        if (mode != 2) {
            double nr = n[0] * r0 + n[1] * r1 + n[2] * r2;
            r0 -= nr * n[0]; r1 -= nr * n[1]; r2 -= nr * n[2];
        }
    } else if (type == 1 && mode != 2) {
        r0 = r1 = r2 = 0.0;
    }
    if (mode >= 1) {
        d4 wi = ld(w + i);
        r0 = wi.x - r0; r1 = wi.y - r1; r2 = wi.z - r2;
        if (type == 1 && mode == 1) r0 = r1 = r2 = 0.0;
    }
    st(out + i, r0, r1, r2);
}

// out = base + D+ w  (base may be null)
__global__ void k_adj_dplus(int n, const d4* __restrict__ dinv, const d4* __restrict__ base,
                            const d4* __restrict__ w, d4* __restrict__ out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    d4 a = ld(dinv + 3 * j), b = ld(dinv + 3 * j + 1), c = ld(dinv + 3 * j + 2), x = ld(w + j);
    double o0 = a.x * x.x + a.y * x.y + a.z * x.z;
    double o1 = b.x * x.x + b.y * x.y + b.z * x.z;
    double o2 = c.x * x.x + c.y * x.y + c.z * x.z;
    if (base) {
        d4 bb = ld(base + j);
        o0 += bb.x; o1 += bb.y; o2 += bb.z;
    }
    st(out + j, o0, o1, o2);
}

// out = base + S_C (L^-T y): backward substitution followed by the projection onto C^T z = 0.
__global__ void k_adj_solve_bwd(DevMesh dm, AdjDev ad, const d4* __restrict__ y, const d4* __restrict__ base,
                                d4* __restrict__ out) {
    int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= dm.m_free) return;
    int lane = threadIdx.x & 31;
    double s0 = 0, s1 = 0, s2 = 0;
    for (int k = dm.kptr[row] + lane; k < dm.kptr[row + 1]; k += 32) {
        double a = dm.kval[k];
        d4 u = ld(y + dm.kidx[k]);
        s0 += a * u.x; s1 += a * u.y; s2 += a * u.z;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane != 0) return;
    int type = ad.type[row];
    if (type == 1) {
        s0 = s1 = s2 = 0.0;
    } else if (type == 2) {
        d4 sl = ld(ad.slip + row), nb = ld(ad.nb + row);
        const double mu = ad.mu[row];
        double cz = (nb.x - mu * sl.x) * s0 + (nb.y - mu * sl.y) * s1 + (nb.z - mu * sl.z) * s2;
        s0 -= cz * nb.x; s1 -= cz * nb.y; s2 -= cz * nb.z;
    }
    d4 bb = ld(base + row);
    st(out + row, bb.x + s0, bb.y + s1, bb.z + s2);
}

// ----------------------------------------------------------------- Krylov helpers
//
// Every vector of the Krylov solve holds the free nodes of all instances (4
// doubles per node).  Reductions are per instance: each instance's segment is
// cut into chunks counted from the instance's own first node, every chunk is
// reduced in a fixed order, and the chunk sums of an instance are added in
// chunk order.  An instance therefore gets bitwise the same dot products alone
// and in any batch.

constexpr int RED_THREADS = 256;
constexpr int DOT_THREADS = 128;

// partial[j * nchunk + c] = sum over chunk c of V_j . w   (grid: chunks x vectors)
__global__ void __launch_bounds__(DOT_THREADS) k_bmdot(const double* __restrict__ V, long ldv,
                                                       const double* __restrict__ w, const int4* __restrict__ chunk,
                                                       int nchunk, double* __restrict__ partial,
                                                       const double* __restrict__ mask,
                                                       const int* __restrict__ clist) {
    __shared__ double sh[DOT_THREADS / 32];
    const int c = clist ? clist[blockIdx.x] : blockIdx.x, j = blockIdx.y;
    const int4 ch = chunk[c];
    if (mask && mask[ch.x] == 0.0) {
        if (threadIdx.x == 0) partial[(long)j * nchunk + c] = 0.0;
        return;
    }
    const double* v = V + j * ldv;
    double s = 0.0;
    for (int i = ch.y + threadIdx.x; i < ch.z; i += DOT_THREADS) s += v[i] * w[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < DOT_THREADS / 32; ++q) t += sh[q];
        partial[(long)j * nchunk + c] = t;
    }
}

// out[j * B + i] = sum of instance i's chunk partials of vector j, in chunk order
__global__ void k_breduce(const double* __restrict__ partial, int nchunk, const int* __restrict__ cptr, int B,
                          int nvec, double* __restrict__ out) {
    int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= B * nvec) return;
    int j = id / B, i = id - j * B;
    const double* p = partial + (long)j * nchunk;
    double s = 0.0;
    for (int c = cptr[i]; c < cptr[i + 1]; ++c) s += p[c];
    out[id] = s;
}

// w += sign * sum_j V_j coef[j * B + inst]   (one block per chunk)
__global__ void k_bvupdate(const double* __restrict__ V, long ldv, int nvec, const double* __restrict__ coef, int B,
                           const int4* __restrict__ chunk, double* __restrict__ w, double sign,
                           const double* __restrict__ mask, const int* __restrict__ clist) {
    const int4 ch = chunk[clist ? clist[blockIdx.x] : blockIdx.x];
    if (mask && mask[ch.x] == 0.0) return;
    for (int i = ch.y + threadIdx.x; i < ch.z; i += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < nvec; ++j) s += V[j * ldv + i] * coef[j * B + ch.x];
        w[i] += sign * s;
    }
}

// out = a * sc[inst]   (one block per chunk)
__global__ void k_bscale(const double* __restrict__ a, const double* __restrict__ sc,
                         const int4* __restrict__ chunk, double* __restrict__ out, const int* __restrict__ clist) {
    const int4 ch = chunk[clist ? clist[blockIdx.x] : blockIdx.x];
    const double f = sc[ch.x];
    for (int i = ch.y + threadIdx.x; i < ch.z; i += blockDim.x) out[i] = f == 0.0 ? 0.0 : a[i] * f;
}

// ----------------------------------------------------------------- gradient outputs

__device__ void normal_jacobian(const DevParams& P, int o, const double x[3], double Dn[9]) {
    for (int q = 0; q < 9; ++q) Dn[q] = 0.0;
    int kind = P.okind[o];
    if (kind == DC_PLANE) return;
    const double* p = P.oprm + 8 * o;
    if (kind == DC_MESH) {
        double nn[3];
        dc_mesh_sdf(P.mesh, (int)p[0], (int)p[1], x, nn, Dn);
        return;
    }
    double c[3];
    double e[3] = {0, 0, 0};
    bool axis = false;
    if (kind == DC_SPHERE) {
        c[0] = p[0]; c[1] = p[1]; c[2] = p[2];
    } else {
        double ab[3] = {p[3] - p[0], p[4] - p[1], p[5] - p[2]};
        double L2 = ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2];
        double t = ((x[0] - p[0]) * ab[0] + (x[1] - p[1]) * ab[1] + (x[2] - p[2]) * ab[2]) / L2;
        if (t <= 0.0) {
            c[0] = p[0]; c[1] = p[1]; c[2] = p[2];
        } else if (t >= 1.0) {
            c[0] = p[3]; c[1] = p[4]; c[2] = p[5];
        } else {
            for (int k = 0; k < 3; ++k) c[k] = p[k] + t * ab[k];
            double L = sqrt(L2);
            for (int k = 0; k < 3; ++k) e[k] = ab[k] / L;
            axis = true;
        }
    }
    double d[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double n[3] = {d[0] / r, d[1] / r, d[2] / r};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double v = (a == b ? 1.0 : 0.0) - n[a] * n[b];
            if (axis) v -= e[a] * e[b];
            Dn[3 * a + b] = v / r;
        }
}

// dL/dx_n = gx - E/h - contact terms (all m nodes); dL/dv_n = M z (free nodes).
// E = h^2 grad^2 W z, resid = g - H z (free nodes; gives the multipliers eta).
__global__ void k_adj_outputs(DevMesh dm, AdjDev ad, DevParams P, const d4* __restrict__ z,
                              const d4* __restrict__ E, const d4* __restrict__ resid, const d4* __restrict__ x_n,
                              const d4* __restrict__ v1, const d4* __restrict__ gx, d4* __restrict__ gx_out,
                              d4* __restrict__ gv_out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= dm.m) return;
    const double h = ad.h;
    d4 g = ld(gx + j), e = ld(E + j);
    double o[3] = {g.x - e.x / h, g.y - e.y / h, g.z - e.z / h};
    if (j >= dm.m_free) {
        st(gx_out + j, o[0], o[1], o[2]);
        st(gv_out + j, 0.0, 0.0, 0.0);
        return;
    }
    d4 zj = ld(z + j);
    double mj = dm.mass[j];
    st(gv_out + j, mj * zj.x, mj * zj.y, mj * zj.z);
    int type = ad.type[j];
    if (type != 0) {
        int ob = ad.contact[j];
        d4 xn = ld(x_n + j), nb = ld(ad.nb + j), r = ld(resid + j);
        double x[3] = {xn.x, xn.y, xn.z}, n[3] = {nb.x, nb.y, nb.z};
        double beta = nb.w;
        double Dn[9];
        normal_jacobian(P, ob, x, Dn);   // symmetric
        if (type == 1) {
            // G_j = v_j + beta n: dG/dx_n = beta Dn + n n^T / h; eta_j = r_j
            double psi[3] = {r.x, r.y, r.z};
            double npsi = n[0] * psi[0] + n[1] * psi[1] + n[2] * psi[2];
            for (int a = 0; a < 3; ++a) {
                double s = 0;
                for (int b = 0; b < 3; ++b) s += Dn[3 * b + a] * psi[b];
                o[a] -= beta * s + n[a] * npsi / h;
            }
        } else {
            // slip: eta_j = n . r_j; G_j = n.v_j + beta; F_j has -h f_N (n - mu t)
            double psi = n[0] * r.x + n[1] * r.y + n[2] * r.z;
            d4 sl = ld(ad.slip + j), vv = ld(v1 + j), ff = ld(ad.f + j);
            double th[3] = {sl.x, sl.y, sl.z};
            double v[3] = {vv.x, vv.y, vv.z};
            double fN = ff.x * n[0] + ff.y * n[1] + ff.z * n[2];
            double vn = n[0] * v[0] + n[1] * v[1] + n[2] * v[2];
            double uT[3] = {v[0] - vn * n[0], v[1] - vn * n[1], v[2] - vn * n[2]};
            double nt = sqrt(uT[0] * uT[0] + uT[1] * uT[1] + uT[2] * uT[2]);
            // dPiv = -((n.v) I + n v^T) Dn ; Dt = (I - t t^T) dPiv / |u_T|
            double M1[9], Dt[9];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double s = 0;
                    for (int c = 0; c < 3; ++c) s += ((a == c ? vn : 0.0) + n[a] * v[c]) * Dn[3 * c + b];
                    M1[3 * a + b] = -s;
                }
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double s = 0;
                    for (int c = 0; c < 3; ++c) s += ((a == c ? 1.0 : 0.0) - th[a] * th[c]) * M1[3 * c + b];
                    Dt[3 * a + b] = s / nt;
                }
            double zz[3] = {zj.x, zj.y, zj.z};
            for (int a = 0; a < 3; ++a) {
                double s = 0, s2 = 0;
                for (int b = 0; b < 3; ++b) {
                    s += (Dn[3 * b + a] - P.node_mu[j] * Dt[3 * b + a]) * zz[b];
                    s2 += Dn[3 * b + a] * v[b];
                }
                o[a] += h * fN * s;
                o[a] -= (s2 + n[a] / h) * psi;
            }
        }
    }
    st(gx_out + j, o[0], o[1], o[2]);
}

// Per-element parameter-gradient terms of one chunk (inst, kind, lo, hi):
// kind 0: -h area_t <A_t z, A_t x - R_t> over triangles t in [lo, hi);
// kind 1: -h a_b <l_b z, q_b - p_b> over bending vertices b in [lo, hi);
// kind 2: -h f_N (t . z_j) over slip nodes j in [lo, hi).   part[c] = chunk sum.
__global__ void k_adj_param_terms(DevMesh dm, AdjDev ad, const d4* __restrict__ z, const d4* __restrict__ x1,
                                  const int4* __restrict__ chunk, double* __restrict__ part) {
    __shared__ double sh[RED_THREADS / 32];
    const double h = ad.h;
    const int4 ch = chunk[blockIdx.x];
    double acc_s = 0.0;
    for (int id = ch.z + threadIdx.x; id < ch.w; id += blockDim.x) {
        if (ch.y == 0) {
            int t = id;
            int4 tr = dm.tri[t];
            d4 g = ld(dm.G + t);
            d4 a = ld(x1 + tr.x), b = ld(x1 + tr.y), c = ld(x1 + tr.z);
            d4 za = ld(z + tr.x), zb = ld(z + tr.y), zc = ld(z + tr.z);
            d4 A0 = ld(ad.tr0 + t), A1 = ld(ad.tr1 + t);
            double acc = 0;
            double xe1[3] = {b.x - a.x, b.y - a.y, b.z - a.z}, xe2[3] = {c.x - a.x, c.y - a.y, c.z - a.z};
            double ze1[3] = {zb.x - za.x, zb.y - za.y, zb.z - za.z}, ze2[3] = {zc.x - za.x, zc.y - za.y, zc.z - za.z};
            double R0[3] = {A0.x, A0.y, A0.z}, R1[3] = {A1.x, A1.y, A1.z};
            for (int k = 0; k < 3; ++k) {
                double F0 = xe1[k] * g.x + xe2[k] * g.z, F1 = xe1[k] * g.y + xe2[k] * g.w;
                double Z0 = ze1[k] * g.x + ze2[k] * g.z, Z1 = ze1[k] * g.y + ze2[k] * g.w;
                acc += Z0 * (F0 - R0[k]) + Z1 * (F1 - R1[k]);
            }
            acc_s -= h * dm.area[t] * acc;
        } else if (ch.y == 1) {
            int b = id;
            double q[3] = {0, 0, 0}, dq[3] = {0, 0, 0};
            for (int k = dm.bptr[b]; k < dm.bptr[b + 1]; ++k) {
                d4 x = ld(x1 + dm.bidx[k]), zz = ld(z + dm.bidx[k]);
                double l = dm.bval[k];
                q[0] += l * x.x; q[1] += l * x.y; q[2] += l * x.z;
                dq[0] += l * zz.x; dq[1] += l * zz.y; dq[2] += l * zz.z;
            }
            double s = dm.sb[b], p[3] = {0, 0, 0};
            if (s > 0.0) {
                double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
                if (nq > 1e-14 * s) {
                    for (int k = 0; k < 3; ++k) p[k] = s * q[k] / nq;
                } else {
                    d4 qr = ld(dm.qrest + b);
                    p[0] = qr.x; p[1] = qr.y; p[2] = qr.z;
                }
            }
            acc_s -= h * dm.abar[b] * (dq[0] * (q[0] - p[0]) + dq[1] * (q[1] - p[1]) + dq[2] * (q[2] - p[2]));
        } else {
            int j = id;
            if (ad.type[j] == 2) {
                d4 sl = ld(ad.slip + j), nb = ld(ad.nb + j), ff = ld(ad.f + j), zj = ld(z + j);
                double fN = ff.x * nb.x + ff.y * nb.y + ff.z * nb.z;
                acc_s -= h * fN * (sl.x * zj.x + sl.y * zj.y + sl.z * zj.z);
            }
        }
    }
    double s = acc_s;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < RED_THREADS / 32; ++k) t += sh[k];
        part[blockIdx.x] = t;
    }
}

// acc[4 i + q] += sum of part over the chunks of (instance i, kind q), in order
__global__ void k_param_accumulate(const double* __restrict__ part, const int* __restrict__ pcptr, int B,
                                   double* __restrict__ acc) {
    int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= 3 * B) return;
    int i = id / 3, q = id - 3 * i;
    double s = 0.0;
    for (int c = pcptr[id]; c < pcptr[id + 1]; ++c) s += part[c];
    acc[4 * i + q] += s;
}

__global__ void k_add_ext(d4* __restrict__ g, const double* __restrict__ ext, const int* __restrict__ int2ext,
                          int m, int cs, long ns) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const long e = (long)int2ext[i] * cs;
    d4 a = ld(g + i);
    st(g + i, a.x + ext[e], a.y + ext[e + ns], a.z + ext[e + 2 * ns]);
}

// rhs = Pi_B (gv + h gx) on free nodes
__global__ void k_adj_rhs(DevMesh dm, AdjDev ad, const d4* __restrict__ gx, const d4* __restrict__ gv,
                          d4* __restrict__ g, d4* __restrict__ rhs) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= dm.m_free) return;
    d4 a = ld(gx + j), b = ld(gv + j);
    double r[3] = {b.x + ad.h * a.x, b.y + ad.h * a.y, b.z + ad.h * a.z};
    st(g + j, r[0], r[1], r[2]);
    int type = ad.type[j];
    if (type == 1) {
        r[0] = r[1] = r[2] = 0.0;
    } else if (type == 2) {
        d4 nb = ld(ad.nb + j);
        double nr = nb.x * r[0] + nb.y * r[1] + nb.z * r[2];
        r[0] -= nr * nb.x; r[1] -= nr * nb.y; r[2] -= nr * nb.z;
    }
    st(rhs + j, r[0], r[1], r[2]);
}

}  // namespace

// ----------------------------------------------------------------- launchers

void adj_setup(const DevMesh& dm, const AdjDev& ad, const d4* x1, const d4* v1, cudaStream_t s) {
    dc_note_launch();
    k_adj_setup_tri<<<nblk(dm.T, 128), 128, 0, s>>>(dm, x1, ad.tr0, ad.tr1, ad.tr2, ad.tav);
    dc_note_launch();
    k_adj_setup_bend<<<nblk(dm.m, 128), 128, 0, s>>>(dm, x1, ad.bq);
    dc_note_launch();
    k_adj_setup_node<<<nblk(dm.m_free, 128), 128, 0, s>>>(dm, ad, v1);
}
void adj_rhs(const DevMesh& dm, const AdjDev& ad, const d4* gx, const d4* gv, d4* g, d4* rhs, cudaStream_t s) {
    dc_note_launch();
    k_adj_rhs<<<nblk(dm.m_free, 128), 128, 0, s>>>(dm, ad, gx, gv, g, rhs);
}
void adj_apply_H(const DevMesh& dm, const AdjDev& ad, int mode, const d4* z, const d4* w, d4* out, cudaStream_t s) {
    dc_note_launch();
    k_adj_elem<<<nblk((long)dm.T + dm.m, dm.bs_elem), dm.bs_elem, 0, s>>>(dm, ad, z, ad.c1, ad.c2, ad.bu);
    int n = (mode == 3) ? dm.m : dm.m_free;
    dc_note_launch();
    k_adj_gather<<<nblk(n, dm.bs_gather), dm.bs_gather, 0, s>>>(dm, ad, mode, z, ad.c1, ad.c2, ad.bu, w, out);
}
void adj_dplus(const DevMesh& dm, const AdjDev& ad, const d4* base, const d4* w, d4* out, cudaStream_t s) {
    dc_note_launch();
    k_adj_dplus<<<nblk(dm.m_free, 128), 128, 0, s>>>(dm.m_free, ad.dinv, base, w, out);
}
void adj_solve_project(const DevMesh& dm, const AdjDev& ad, const d4* r, d4* ytmp, const d4* base, d4* out,
                       cudaStream_t s) {
    launch_solve_fwd(dm, r, ytmp, s);
    dc_note_launch();
    k_adj_solve_bwd<<<nblk((long)dm.m_free * 32, 256), 256, 0, s>>>(dm, ad, ytmp, base, out);
}
void adj_bdot(const Segs& sg, const double* V, long ldv, int nvec, const double* w, double* partial, double* out,
              cudaStream_t s, const double* mask, const int* clist, int ncl) {
    if (clist && ncl == 0) return;
    dc_note_launch();
    k_bmdot<<<dim3(clist ? ncl : sg.nchunk, nvec), DOT_THREADS, 0, s>>>(V, ldv, w, sg.chunk, sg.nchunk, partial, mask,
                                                                        clist);
    dc_note_launch();
    k_breduce<<<nblk((long)sg.B * nvec, 128), 128, 0, s>>>(partial, sg.nchunk, sg.cptr, sg.B, nvec, out);
}
void adj_bvupdate(const Segs& sg, const double* V, long ldv, int nvec, const double* coef, double* w, double sign,
                  cudaStream_t s, const double* mask, const int* clist, int ncl) {
    if (clist && ncl == 0) return;
    dc_note_launch();
    k_bvupdate<<<clist ? ncl : sg.nchunk, 128, 0, s>>>(V, ldv, nvec, coef, sg.B, sg.chunk, w, sign, mask, clist);
}
void adj_bscale(const Segs& sg, const double* a, const double* sc, double* out, cudaStream_t s, const int* clist,
                int ncl) {
    if (clist && ncl == 0) return;
    dc_note_launch();
    k_bscale<<<clist ? ncl : sg.nchunk, 128, 0, s>>>(a, sc, sg.chunk, out, clist);
}
void adj_outputs(const DevMesh& dm, const AdjDev& ad, const DevParams& P, const d4* z, const d4* E,
                 const d4* resid, const d4* x_n, const d4* v1, const d4* gx, d4* gx_out, d4* gv_out,
                 cudaStream_t s) {
    dc_note_launch();
    k_adj_outputs<<<nblk(dm.m, 128), 128, 0, s>>>(dm, ad, P, z, E, resid, x_n, v1, gx, gx_out, gv_out);
}
void adj_params(const DevMesh& dm, const AdjDev& ad, const Segs& sg, const d4* z, const d4* x1, double* part,
                double* acc, cudaStream_t s) {
    dc_note_launch();
    k_adj_param_terms<<<sg.npchunk, RED_THREADS, 0, s>>>(dm, ad, z, x1, sg.pchunk, part);
    dc_note_launch();
    k_param_accumulate<<<nblk(3L * sg.B, 128), 128, 0, s>>>(part, sg.pcptr, sg.B, acc);
}
void adj_add_ext(d4* g, const double* ext, const int* int2ext, int m, int layout, cudaStream_t s) {
    const bool cm = layout == DC_LAYOUT_COMPONENT_MAJOR;
    dc_note_launch();
    k_add_ext<<<nblk(m, 256), 256, 0, s>>>(g, ext, int2ext, m, cm ? 1 : 3, cm ? (long)m : 1L);
}
