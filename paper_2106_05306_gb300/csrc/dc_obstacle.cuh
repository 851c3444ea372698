// Signed distance, normal and normal Jacobian of a closed triangle-mesh obstacle
// (DC_MESH), shared by contact detection and the adjoint.  Reading of Sec. 3.2
// ("Extensions": any obstacle with a signed distance) and of the paper's
// remarks on triangulated obstacles (Sec. "Continuity and Smoothness").
//
// A mesh is a run of triangle records of DC_MESH_REC d4 each:
//   [0..2] vertices A, B, C; [3] unit face normal; [4..6] pseudo-normals of the
//   edges AB, BC, CA (sum of the two incident face normals); [7..9]
//   angle-weighted pseudo-normals of the vertices A, B, C.
// phi(x) = s |x - c| with c the closest surface point and s the sign of
// (x - c) . N for the pseudo-normal N of c's feature (face, edge or vertex);
// n = grad phi = s (x - c)/|x - c|.  Triangles whose distance is within
// DC_MESH_TIE (relative, plus DC_MESH_TIE_ABS) of the smallest tie, and the lowest
// index among them wins, so that points equidistant from several faces are not
// decided by rounding.  Closer than DC_MESH_ON_SURFACE metres (where a stick or
// slip step leaves a node, and x - c is rounding) the point is on the surface and
// n = N/|N| for the pseudo-normal N of the feature c lies on to within
// DC_MESH_SNAP metres: the first vertex A, B, C, else the first edge AB, BC, CA,
// else the face.  The Hessian of phi is 0 in a face region and on the surface,
// s (I - u u^T - e e^T)/r on an edge (e its unit direction) and s (I - u u^T)/r at
// a vertex, u = (x - c)/r, r = |x - c|.
#pragma once

constexpr int DC_MESH_REC = 10;
constexpr double DC_MESH_TIE = 1e-9;
constexpr double DC_MESH_TIE_ABS = 1e-14;
constexpr double DC_MESH_ON_SURFACE = 1e-12;
constexpr double DC_MESH_SNAP = 1e-9;

// Closest point q of triangle (a, b, c) to p, by the Voronoi-region tests of
// Ericson ("Real-Time Collision Detection", Sec. 5.1.5).  Returns the feature:
// 0 face, 1 edge AB, 2 edge BC, 3 edge CA, 4 vertex A, 5 vertex B, 6 vertex C.
__device__ __forceinline__ int dc_closest_on_triangle(const double p[3], const double a[3], const double b[3],
                                                      const double c[3], double q[3]) {
    double ab[3], ac[3], ap[3];
    for (int k = 0; k < 3; ++k) { ab[k] = b[k] - a[k]; ac[k] = c[k] - a[k]; ap[k] = p[k] - a[k]; }
    const double d1 = ab[0] * ap[0] + ab[1] * ap[1] + ab[2] * ap[2];
    const double d2 = ac[0] * ap[0] + ac[1] * ap[1] + ac[2] * ap[2];
    if (d1 <= 0.0 && d2 <= 0.0) {
        for (int k = 0; k < 3; ++k) q[k] = a[k];
        return 4;
    }
    double bp[3] = {p[0] - b[0], p[1] - b[1], p[2] - b[2]};
    const double d3 = ab[0] * bp[0] + ab[1] * bp[1] + ab[2] * bp[2];
    const double d4v = ac[0] * bp[0] + ac[1] * bp[1] + ac[2] * bp[2];
    if (d3 >= 0.0 && d4v <= d3) {
        for (int k = 0; k < 3; ++k) q[k] = b[k];
        return 5;
    }
    const double vc = d1 * d4v - d3 * d2;
    if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
        const double v = d1 / (d1 - d3);
        for (int k = 0; k < 3; ++k) q[k] = a[k] + v * ab[k];
        return 1;
    }
    double cp[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
    const double d5 = ab[0] * cp[0] + ab[1] * cp[1] + ab[2] * cp[2];
    const double d6 = ac[0] * cp[0] + ac[1] * cp[1] + ac[2] * cp[2];
    if (d6 >= 0.0 && d5 <= d6) {
        for (int k = 0; k < 3; ++k) q[k] = c[k];
        return 6;
    }
    const double vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
        const double w = d2 / (d2 - d6);
        for (int k = 0; k < 3; ++k) q[k] = a[k] + w * ac[k];
        return 3;
    }
    const double va = d3 * d6 - d5 * d4v;
    if (va <= 0.0 && (d4v - d3) >= 0.0 && (d5 - d6) >= 0.0) {
        const double w = (d4v - d3) / ((d4v - d3) + (d5 - d6));
        for (int k = 0; k < 3; ++k) q[k] = b[k] + w * (c[k] - b[k]);
        return 2;
    }
    const double den = 1.0 / (va + vb + vc);
    const double v = vb * den, w = vc * den;
    for (int k = 0; k < 3; ++k) q[k] = a[k] + ab[k] * v + ac[k] * w;
    return 0;
}

// phi of mesh triangles rec[t0 .. t0 + nt) at x; n (if not null) receives
// grad phi and Dn (if not null) the 3x3 Jacobian of n, row-major.
__device__ inline double dc_mesh_sdf(const d4* __restrict__ rec, int t0, int nt, const double x[3], double* n,
                                     double* Dn) {
    // pass 1: the smallest distance; pass 2: the lowest triangle within the tie band
    auto closest = [&](int t, double q[3]) {
        const d4* r = rec + (long)t * DC_MESH_REC;
        const double a[3] = {r[0].x, r[0].y, r[0].z}, b[3] = {r[1].x, r[1].y, r[1].z},
                     c[3] = {r[2].x, r[2].y, r[2].z};
        return dc_closest_on_triangle(x, a, b, c, q);
    };
    double dmin = 1e300;
    for (int t = t0; t < t0 + nt; ++t) {
        double q[3];
        closest(t, q);
        const double dx = x[0] - q[0], dy = x[1] - q[1], dz = x[2] - q[2];
        dmin = fmin(dmin, sqrt(dx * dx + dy * dy + dz * dz));
    }
    double best = 0.0, cbest[3] = {0, 0, 0};
    int tb = -1, fb = 0;
    const double band = dmin * (1.0 + DC_MESH_TIE) + DC_MESH_TIE_ABS;
    for (int t = t0; t < t0 + nt && tb < 0; ++t) {
        double q[3];
        const int f = closest(t, q);
        const double dx = x[0] - q[0], dy = x[1] - q[1], dz = x[2] - q[2];
        const double d = sqrt(dx * dx + dy * dy + dz * dz);
        if (d <= band) {
            best = d;
            tb = t;
            fb = f;
            cbest[0] = q[0]; cbest[1] = q[1]; cbest[2] = q[2];
        }
    }
    if (Dn)
        for (int k = 0; k < 9; ++k) Dn[k] = 0.0;
    if (tb < 0) {
        if (n) { n[0] = 0.0; n[1] = 1.0; n[2] = 0.0; }
        return 1e300;
    }
    const d4* r = rec + (long)tb * DC_MESH_REC;
    const d4 N = r[3 + fb];   // face normal (3), edge (4..6) or vertex (7..9) pseudo-normal
    const double u[3] = {x[0] - cbest[0], x[1] - cbest[1], x[2] - cbest[2]};
    const double s = (u[0] * N.x + u[1] * N.y + u[2] * N.z) >= 0.0 ? 1.0 : -1.0;
    const double rr = best;
    if (rr < DC_MESH_ON_SURFACE) {
        if (n) {
            int feat = 0;   // record slot offset: 0 face, 1..3 edges, 4..6 vertices
            for (int k = 0; k < 3 && !feat; ++k) {
                const double dx = cbest[0] - r[k].x, dy = cbest[1] - r[k].y, dz = cbest[2] - r[k].z;
                if (sqrt(dx * dx + dy * dy + dz * dz) <= DC_MESH_SNAP) feat = 4 + k;
            }
            for (int k = 0; k < 3 && !feat; ++k) {
                const d4 a = r[k], b = r[(k + 1) % 3];
                const double e[3] = {b.x - a.x, b.y - a.y, b.z - a.z};
                const double w[3] = {cbest[0] - a.x, cbest[1] - a.y, cbest[2] - a.z};
                const double t = fmin(fmax((w[0] * e[0] + w[1] * e[1] + w[2] * e[2]) /
                                               (e[0] * e[0] + e[1] * e[1] + e[2] * e[2]), 0.0), 1.0);
                const double dx = w[0] - t * e[0], dy = w[1] - t * e[1], dz = w[2] - t * e[2];
                if (sqrt(dx * dx + dy * dy + dz * dz) <= DC_MESH_SNAP) feat = 1 + k;
            }
            const d4 Ns = r[3 + feat];
            const double iN = 1.0 / sqrt(Ns.x * Ns.x + Ns.y * Ns.y + Ns.z * Ns.z);
            n[0] = Ns.x * iN; n[1] = Ns.y * iN; n[2] = Ns.z * iN;
        }
        return s * rr;
    }
    const double iu = 1.0 / rr;
    const double un[3] = {u[0] * iu, u[1] * iu, u[2] * iu};
    if (n) { n[0] = s * un[0]; n[1] = s * un[1]; n[2] = s * un[2]; }
    if (Dn && fb != 0) {
        double e[3] = {0.0, 0.0, 0.0};
        if (fb <= 3) {   // edge AB, BC or CA
            const d4 P0 = r[fb - 1], P1 = r[fb % 3];
            double ed[3] = {P1.x - P0.x, P1.y - P0.y, P1.z - P0.z};
            const double ie = 1.0 / sqrt(ed[0] * ed[0] + ed[1] * ed[1] + ed[2] * ed[2]);
            e[0] = ed[0] * ie; e[1] = ed[1] * ie; e[2] = ed[2] * ie;
        }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                Dn[3 * a + b] = s * ((a == b ? 1.0 : 0.0) - un[a] * un[b] - e[a] * e[b]) * iu;
    }
    return s * rr;
}
