// Polar factor of a triangle's 3x2 deformation gradient (reading R1 of the
// stretch energy, Eq. pd_project: the projection onto matrices with
// orthonormal columns), shared by the forward local step and the adjoint setup.
#pragma once

// F and R are column-major: F[0..2] is column f0, F[3..5] column f1.
//
// Regular case, det C > 1e-30 (tr C)^2 with C = F^T F: the closed form
//   S = (C + s I) / t,  s = sqrt(det C) = |f0 x f1|,  t = sqrt(tr C + 2 s),
//   R = F S^-1 = F adj(C + s I) / (s t),
// with s from the cross product (Lagrange's identity), which stays exact for
// a triangle collapsed onto a line.  sinv receives S^-1 (s00, s01, s11) and
// *itr = 1 / tr S = 1 / t.
//
// Collapsed case (F of rank <= 1, no unique polar factor): v1 is the unit
// eigenvector of C of its larger eigenvalue, v2 = v1 turned by +90 degrees,
// u1 = F v1 / |F v1|, u2 = normalize(u1 x e_a) with e_a the first coordinate
// axis (x, y, z order) with |u1_a| <= 0.6 (one exists since 1/sqrt(3) < 0.6, and
// the choice is stable against rounding noise in the components of an
// axis-aligned u1), and R = u1 v1^T + u2 v2^T; F = 0 gives
// R = [e_x, e_y].  The projection is taken as locally constant there, so S^-1
// and 1/tr S are returned as 0 (no polar-derivative term in the adjoint).
// Returns true in the collapsed case.
__device__ __forceinline__ bool dc_polar3x2(const double F[6], double R[6], double sinv[3], double* itr) {
    const double c00 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
    const double c01 = F[0] * F[3] + F[1] * F[4] + F[2] * F[5];
    const double c11 = F[3] * F[3] + F[4] * F[4] + F[5] * F[5];
    const double cx = F[1] * F[5] - F[2] * F[4];
    const double cy = F[2] * F[3] - F[0] * F[5];
    const double cz = F[0] * F[4] - F[1] * F[3];
    const double det = cx * cx + cy * cy + cz * cz;
    const double tr = c00 + c11;
    if (det > 1e-30 * tr * tr) {
        const double is = rsqrt(det);
        const double s = det * is;
        const double it = rsqrt(tr + 2.0 * s);
        const double k = is * it;
        const double a = (c11 + s) * k, b = -c01 * k, d = (c00 + s) * k;   // S^-1
        R[0] = a * F[0] + b * F[3]; R[1] = a * F[1] + b * F[4]; R[2] = a * F[2] + b * F[5];
        R[3] = b * F[0] + d * F[3]; R[4] = b * F[1] + d * F[4]; R[5] = b * F[2] + d * F[5];
        sinv[0] = a; sinv[1] = b; sinv[2] = d;
        *itr = it;
        return false;
    }
    sinv[0] = sinv[1] = sinv[2] = 0.0;
    *itr = 0.0;
    if (tr == 0.0) {
        R[0] = 1.0; R[1] = 0.0; R[2] = 0.0;
        R[3] = 0.0; R[4] = 1.0; R[5] = 0.0;
        return true;
    }
    const double dd = 0.5 * (c00 - c11);
    const double r = hypot(dd, c01);
    double v0, v1;
    if (dd >= 0.0) { v0 = dd + r; v1 = c01; }
    else { v0 = c01; v1 = r - dd; }
    const double nv = 1.0 / sqrt(v0 * v0 + v1 * v1);
    v0 *= nv;
    v1 *= nv;
    double u[3] = {F[0] * v0 + F[3] * v1, F[1] * v0 + F[4] * v1, F[2] * v0 + F[5] * v1};
    const double nu = 1.0 / sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    u[0] *= nu; u[1] *= nu; u[2] *= nu;
    double w[3];
    if (fabs(u[0]) <= 0.6) { w[0] = 0.0; w[1] = u[2]; w[2] = -u[1]; }          // u1 x e_x
    else if (fabs(u[1]) <= 0.6) { w[0] = -u[2]; w[1] = 0.0; w[2] = u[0]; }     // u1 x e_y
    else { w[0] = u[1]; w[1] = -u[0]; w[2] = 0.0; }                             // u1 x e_z
    const double nw = 1.0 / sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    w[0] *= nw; w[1] *= nw; w[2] *= nw;
    // R = u1 v1^T + u2 v2^T with v1 = (v0, v1), v2 = (-v1, v0)
    for (int c = 0; c < 3; ++c) {
        R[c] = u[c] * v0 - w[c] * v1;
        R[3 + c] = u[c] * v1 + w[c] * v0;
    }
    return true;
}
