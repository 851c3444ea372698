// Forward-step kernels of libdc (FP64, sm_103a).
//
// One PD iteration (Sec. 3.1-3.2) is four launches:
//   local   -- per triangle: polar projection of F (stretch) and its right-hand
//              side contribution; per vertex: bending projection;
//   gather  -- per free node: b = M (v_n + h g) + h sum_i w_i A_i^T (p_i - A_i x_n)
//              + h f   (Eq. pd_velocity / pd_velocity_with_contact, expanded so
//              that the O(h^2 |L x|) terms never cancel);
//   solve_fwd / solve_bwd -- v_half = L^-T L^-1 b with the explicit inverse
//              factor, and the per-node Signorini-Coulomb update fused into the
//              backward sweep (Eq. contact_all).
// Every reduction is a fixed-order gather (no atomics), so a launch is bitwise
// repeatable and independent of what else runs on the GPU.
#include <algorithm>
#include <atomic>
#include <mutex>

#include "dc_internal.h"
#include "dc_obstacle.cuh"
#include "dc_polar.cuh"
#include "dc_wait.cuh"

namespace {
std::atomic<long long> g_launches{0};
}  // namespace

void dc_note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void dc_add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long dc_launch_count() { return g_launches.load(std::memory_order_relaxed); }

namespace {

__device__ __forceinline__ d4 ld(const d4* p) {
    const double2* q = reinterpret_cast<const double2*>(p);
    double2 a = q[0], b = q[1];
    d4 r;
    r.x = a.x; r.y = a.y; r.z = b.x; r.w = b.y;
    return r;
}
// a load through L2 only, for data that other CTAs of the same launch write
__device__ __forceinline__ d4 ld_cg(const d4* p) {
    const double2* q = reinterpret_cast<const double2*>(p);
    double2 a = __ldcg(q), b = __ldcg(q + 1);
    d4 r;
    r.x = a.x; r.y = a.y; r.z = b.x; r.w = b.y;
    return r;
}
__device__ __forceinline__ void st(d4* p, double x, double y, double z, double w = 0.0) {
    double2* q = reinterpret_cast<double2*>(p);
    q[0] = make_double2(x, y);
    q[1] = make_double2(z, w);
}

// Signed distance and its gradient for one analytic obstacle (reading R4).
__device__ double sdf(const DevParams& P, int o, double x, double y, double z, double* n) {
    const double* q = P.oprm + 8 * o;
    const int kind = P.okind[o];
    if (kind == DC_MESH) {
        const double xx[3] = {x, y, z};
        return dc_mesh_sdf(P.mesh, (int)q[0], (int)q[1], xx, n, nullptr);
    }
    if (kind == DC_PLANE) {
        if (n) { n[0] = q[0]; n[1] = q[1]; n[2] = q[2]; }
        return q[0] * x + q[1] * y + q[2] * z - q[3];
    }
    double cx, cy, cz, r;
    if (kind == DC_SPHERE) {
        cx = q[0]; cy = q[1]; cz = q[2]; r = q[3];
    } else {
        double abx = q[3] - q[0], aby = q[4] - q[1], abz = q[5] - q[2];
        double t = ((x - q[0]) * abx + (y - q[1]) * aby + (z - q[2]) * abz) /
                   (abx * abx + aby * aby + abz * abz);
        t = fmin(fmax(t, 0.0), 1.0);
        cx = q[0] + t * abx; cy = q[1] + t * aby; cz = q[2] + t * abz; r = q[6];
    }
    double dx = x - cx, dy = y - cy, dz = z - cz;
    double d = sqrt(dx * dx + dy * dy + dz * dz);
    if (n) { n[0] = dx / d; n[1] = dy / d; n[2] = dz / d; }
    return d - r;
}

// Boundary arrays: component c of caller node e sits at ext[e * cs + c * ns]
// with (cs, ns) = (3, 1) node-major ([m][3]) or (1, m) component-major ([3][m]).
__global__ void k_permute_in(const double* __restrict__ ext, d4* __restrict__ out,
                             const int* __restrict__ int2ext, int m, int cs, long ns) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const long e = (long)int2ext[i] * cs;
    st(out + i, ext[e], ext[e + ns], ext[e + 2 * ns]);
}

__global__ void k_permute_out(const d4* __restrict__ in, double* __restrict__ ext,
                              const int* __restrict__ int2ext, int m, int cs, long ns) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const long e = (long)int2ext[i] * cs;
    d4 a = ld(in + i);
    ext[e] = a.x; ext[e + ns] = a.y; ext[e + 2 * ns] = a.z;
}

__global__ void k_zero_range(d4* v, int lo, int hi) {
    int i = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (i < hi) st(v + i, 0.0, 0.0, 0.0);
}

// Contact set, normal and bias for the step (reading R4); resets the impulse.
__global__ void k_detect(DevMesh dm, DevParams P, const d4* __restrict__ x_n, const d4* __restrict__ v_n,
                         int* __restrict__ contact, d4* __restrict__ nb, d4* __restrict__ f,
                         d4* __restrict__ ind) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dm.m_free) return;
    d4 x = ld(x_n + i), v = ld(v_n + i);
    double px = x.x + P.h * v.x, py = x.y + P.h * v.y, pz = x.z + P.h * v.z;
    double best = 1e300;
    int bo = -1;
    const int inst = P.node_inst[i];
    for (int o = P.optr[inst]; o < P.optr[inst + 1]; ++o) {
        double ph = sdf(P, o, px, py, pz, nullptr);
        if (ph < best) { best = ph; bo = o; }
    }
    st(f + i, 0.0, 0.0, 0.0);
    if (bo >= 0 && best <= P.delta) {
        double n[3];
        double ph0 = sdf(P, bo, x.x, x.y, x.z, n);
        contact[i] = bo;
        st(nb + i, n[0], n[1], n[2], ph0 / P.h);
        st(ind + i, 1.0, 1.0, 1.0);
    } else {
        contact[i] = -1;
        st(ind + i, 0.0, 0.0, 0.0);
    }
}

// Polar factor R of a 3x2 F (reading R1): the closed form, or the fixed rule
// for a triangle collapsed onto a line (dc_polar.cuh).
__device__ __forceinline__ void polar3x2(const double F[6], double R[6]) {
    double sinv[3], itr;
    dc_polar3x2(F, R, sinv, &itr);
}

// Local step.  Threads [0, T): triangles; [T, T + m): bending vertices.
__global__ void k_local(DevMesh dm, DevParams P, const d4* __restrict__ x_n, const d4* __restrict__ v,
                        d4* __restrict__ c1, d4* __restrict__ c2, d4* __restrict__ bu) {
    int id = blockIdx.x * blockDim.x + threadIdx.x;
    const double h = P.h;
    if (id < dm.T) {
        int4 tr = dm.tri[id];
        d4 g = ld(dm.G + id);
        double w = dm.wt[id] * h;
        d4 x0 = ld(x_n + tr.x), x1 = ld(x_n + tr.y), x2 = ld(x_n + tr.z);
        d4 v0 = ld(v + tr.x), v1 = ld(v + tr.y), v2 = ld(v + tr.z);
        double e1[3] = {x1.x - x0.x, x1.y - x0.y, x1.z - x0.z};
        double e2[3] = {x2.x - x0.x, x2.y - x0.y, x2.z - x0.z};
        double f1[3] = {v1.x - v0.x, v1.y - v0.y, v1.z - v0.z};
        double f2[3] = {v2.x - v0.x, v2.y - v0.y, v2.z - v0.z};
        double Fn[6], F[6], R[6];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Fn[c] = e1[c] * g.x + e2[c] * g.z;          // column 0
            Fn[3 + c] = e1[c] * g.y + e2[c] * g.w;      // column 1
            F[c] = Fn[c] + h * (f1[c] * g.x + f2[c] * g.z);
            F[3 + c] = Fn[3 + c] + h * (f1[c] * g.y + f2[c] * g.w);
        }
        polar3x2(F, R);
        // p - A x_n (Eq. pd_velocity), or p - A x^k for the mass splitting
        const double* Fr = P.mass_split ? F : Fn;
        double D[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) D[k] = w * (R[k] - Fr[k]);
        st(c1 + id, D[0] * g.x + D[3] * g.y, D[1] * g.x + D[4] * g.y, D[2] * g.x + D[5] * g.y);
        st(c2 + id, D[0] * g.z + D[3] * g.w, D[1] * g.z + D[4] * g.w, D[2] * g.z + D[5] * g.w);
        return;
    }
    int b = id - dm.T;
    if (b >= dm.m) return;
    double qn[3] = {0, 0, 0}, qv[3] = {0, 0, 0};
    for (int k = dm.bptr[b]; k < dm.bptr[b + 1]; ++k) {
        int j = dm.bidx[k];
        double l = dm.bval[k];
        d4 xj = ld(x_n + j), vj = ld(v + j);
        qn[0] += l * xj.x; qn[1] += l * xj.y; qn[2] += l * xj.z;
        qv[0] += l * vj.x; qv[1] += l * vj.y; qv[2] += l * vj.z;
    }
    double q[3] = {qn[0] + h * qv[0], qn[1] + h * qv[1], qn[2] + h * qv[2]};
    double s = dm.sb[b];
    double p[3] = {0, 0, 0};
    if (s > 0.0) {
        double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
        if (nq > 1e-14 * s) {
            double k = s / nq;
            p[0] = k * q[0]; p[1] = k * q[1]; p[2] = k * q[2];
        } else {
            d4 qr = ld(dm.qrest + b);
            p[0] = qr.x; p[1] = qr.y; p[2] = qr.z;
        }
    }
    double w = dm.wb[b] * h;
    const double* qr = P.mass_split ? q : qn;
    st(bu + b, w * (p[0] - qr[0]), w * (p[1] - qr[1]), w * (p[2] - qr[2]));
}

__global__ void k_gather_rhs(DevMesh dm, DevParams P, const d4* __restrict__ v_n, const d4* __restrict__ c1,
                             const d4* __restrict__ c2, const d4* __restrict__ bu, const d4* __restrict__ f,
                             d4* __restrict__ b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dm.m_free) return;
    d4 vn = ld(v_n + i);
    double mi = dm.mass[i];
    double r0 = mi * (vn.x + P.h * P.g[0]);
    double r1 = mi * (vn.y + P.h * P.g[1]);
    double r2 = mi * (vn.z + P.h * P.g[2]);
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
    d4 fi = ld(f + i);
    st(b + i, r0 + P.h * fi.x, r1 + P.h * fi.y, r2 + P.h * fi.z);
}

// y_i = sum_k Linv(i,k) b_k, one warp per row, fixed lane order.
__device__ __forceinline__ void warp_row(const int* __restrict__ ptr, const int* __restrict__ idx,
                                         const double* __restrict__ val, const d4* __restrict__ in, int row,
                                         double& s0, double& s1, double& s2) {
    int lane = threadIdx.x & 31;
    s0 = s1 = s2 = 0.0;
    for (int k = ptr[row] + lane; k < ptr[row + 1]; k += 32) {
        double a = val[k];
        d4 u = ld(in + idx[k]);
        s0 += a * u.x; s1 += a * u.y; s2 += a * u.z;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
}

// Forward substitution with the explicit inverse factor, y = L^-1 b.  Rows with
// more than LONG_ROW nonzeros (separator rows near the top of the elimination
// tree) get a whole CTA each; the other rows one warp each.  Both reductions
// run in a fixed order, so the result is bitwise repeatable.
__global__ void __launch_bounds__(256) k_solve_fwd(DevMesh dm, const d4* __restrict__ b, d4* __restrict__ y) {
    __shared__ double red[3][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if ((int)blockIdx.x < dm.n_long) {
        const int row = dm.long_rows[blockIdx.x];
        double s0 = 0, s1 = 0, s2 = 0;
        const int lo = dm.fptr[row], hi = dm.fptr[row + 1];
        int k = lo + threadIdx.x;
        for (; k + 256 < hi; k += 512) {
            const double a0 = dm.fval[k], a1 = dm.fval[k + 256];
            const d4 u0 = ld(b + dm.fidx[k]), u1 = ld(b + dm.fidx[k + 256]);
            s0 += a0 * u0.x + a1 * u1.x; s1 += a0 * u0.y + a1 * u1.y; s2 += a0 * u0.z + a1 * u1.z;
        }
        if (k < hi) {
            const double a = dm.fval[k];
            const d4 u = ld(b + dm.fidx[k]);
            s0 += a * u.x; s1 += a * u.y; s2 += a * u.z;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) { red[0][warp] = s0; red[1][warp] = s1; red[2][warp] = s2; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t0 = 0, t1 = 0, t2 = 0;
            for (int w = 0; w < 8; ++w) { t0 += red[0][w]; t1 += red[1][w]; t2 += red[2][w]; }
            st(y + row, t0, t1, t2);
        }
        return;
    }
    const int q = ((int)blockIdx.x - dm.n_long) * 8 + warp;
    if (q >= dm.n_short) return;
    const int row = dm.short_rows[q];
    double s0 = 0, s1 = 0, s2 = 0;
    const int lo = dm.fptr[row], hi = dm.fptr[row + 1];
    int k = lo + lane;
    for (; k + 32 < hi; k += 64) {
        const double a0 = dm.fval[k], a1 = dm.fval[k + 32];
        const d4 u0 = ld(b + dm.fidx[k]), u1 = ld(b + dm.fidx[k + 32]);
        s0 += a0 * u0.x + a1 * u1.x; s1 += a0 * u0.y + a1 * u1.y; s2 += a0 * u0.z + a1 * u1.z;
    }
    if (k < hi) {
        const double a = dm.fval[k];
        const d4 u = ld(b + dm.fidx[k]);
        s0 += a * u.x; s1 += a * u.y; s2 += a * u.z;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) st(y + row, s0, s1, s2);
}

// Per-node Signorini-Coulomb solve (Eq. contact_1-3, reading R5) in world
// frame: v = vt + c f, u_N = n.v + beta, u_T = v - (n.v) n.
__device__ __forceinline__ int coulomb(double mu, double c, const double n[3], double beta,
                                       const double vt[3], double v[3], double f[3]) {
    double vn = n[0] * vt[0] + n[1] * vt[1] + n[2] * vt[2];
    double uN = vn + beta;
    if (uN >= 0.0) {                                        // take off
        v[0] = vt[0]; v[1] = vt[1]; v[2] = vt[2];
        f[0] = f[1] = f[2] = 0.0;
        return 0;
    }
    double uT[3] = {vt[0] - vn * n[0], vt[1] - vn * n[1], vt[2] - vn * n[2]};
    double nt = sqrt(uT[0] * uT[0] + uT[1] * uT[1] + uT[2] * uT[2]);
    if (nt <= mu * (-uN)) {                                 // stick
        for (int k = 0; k < 3; ++k) {
            v[k] = -beta * n[k];
            f[k] = (v[k] - vt[k]) / c;
        }
        return 1;
    }
    double fN = -uN / c;                                    // slip
    double ft = mu * fN / nt;
    for (int k = 0; k < 3; ++k) {
        f[k] = fN * n[k] - ft * uT[k];
        v[k] = vt[k] + c * f[k];
    }
    return 2;
}

// Output of one row of the backward substitution: mode 0 stores it; mode 1
// applies the node's Signorini-Coulomb update (contact nodes) and stores v; mode 2
// stores the compliance c_j = h s0.
__device__ __forceinline__ void finish_row(const DevParams& P, int row, double s0, double s1, double s2,
                                           d4* __restrict__ out, int mode, const int* __restrict__ contact,
                                           const d4* __restrict__ nb, const double* __restrict__ cc,
                                           d4* __restrict__ f, int* __restrict__ case_, double* __restrict__ c_out) {
    if (mode == 2) {
        c_out[row] = P.h * s0;
        return;
    }
    if (mode == 1 && contact[row] >= 0) {
        d4 q = ld(nb + row), fo = ld(f + row);
        double c = cc[row];
        double n[3] = {q.x, q.y, q.z};
        double vt[3] = {s0 - c * fo.x, s1 - c * fo.y, s2 - c * fo.z};
        double v[3], fn[3];
        case_[row] = coulomb(P.node_mu[row], c, n, q.w, vt, v, fn);
        st(f + row, fn[0], fn[1], fn[2]);
        st(out + row, v[0], v[1], v[2]);
        return;
    }
    st(out + row, s0, s1, s2);
}

__global__ void k_solve_bwd(DevMesh dm, DevParams P, const d4* __restrict__ y, d4* __restrict__ out, int mode,
                            const int* __restrict__ contact, const d4* __restrict__ nb,
                            const double* __restrict__ cc, d4* __restrict__ f, int* __restrict__ case_,
                            double* __restrict__ c_out) {
    int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= dm.m_free) return;
    double s0, s1, s2;
    warp_row(dm.kptr, dm.kidx, dm.kval, y, row, s0, s1, s2);
    if ((threadIdx.x & 31) != 0) return;
    finish_row(P, row, s0, s1, s2, out, mode, contact, nb, cc, f, case_, c_out);
}

// Issues L2 prefetches for [p, p + bytes) (128-byte lines, spread over the CTA),
// so that a front's blocks stream in from HBM while the CTA gathers its inputs.
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
    const char* c = static_cast<const char*>(p);
    for (size_t o = (size_t)threadIdx.x * 128; o < bytes; o += (size_t)blockDim.x * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(c + o));
}

// ---- supernodal substitution (global_solver 1): one CTA per supernode, levels
// leaves-first for L y = b and root-first for L^T x = y, three right-hand sides.
// Shared memory holds the front's vectors component-major ([3][n]).

// Column-major product on one CTA with three right-hand sides: t_c,i = sum_k
// A[k * lda + i] v[c * ldv + k] for i < nrows and k < K (tri 1: only k <= i;
// tri 2: only k >= i).  Rows go in passes of GV_ROWS; the k range is cut into G
// contiguous chunks with G a function of K alone.  Every (row, chunk) pair with
// a nonempty k range is one work item -- the pairs are numbered chunk by chunk,
// so that the triangle's empty pairs take no lanes -- and a row's partial sums
// are added in chunk order.  The result depends only on (nrows, K), never on the
// CTA size (a supernode gives the same bits whatever else shares its launch).
// fin(i, t0, t1, t2) stores (it must not write v).
constexpr int GV_ROWS = 128;
constexpr int GV_MAXG = 8;
__host__ __device__ constexpr int gv_groups(int K) { return K <= 8 ? 1 : (K + 7) / 8 < GV_MAXG ? (K + 7) / 8 : GV_MAXG; }

template <class Fin>
__device__ __forceinline__ void cm_gemv3(const double* __restrict__ A, long lda, int nrows, int K, int tri,
                                         const double* __restrict__ v, int ldv, double* __restrict__ red, Fin fin) {
    const int nt = blockDim.x, tid = threadIdx.x;
    const int G = gv_groups(K);
    const int C = (K + G - 1) / G;
    constexpr int RS = GV_ROWS * GV_MAXG;      // stride between the three columns' partial sums
    for (int i0 = 0; i0 < nrows; i0 += GV_ROWS) {
        const int R = min(GV_ROWS, nrows - i0);
        // rows [lo(g), hi(g)) of this pass have a nonempty k range in chunk g
        auto lo = [&](int g) { return tri == 1 ? min(R, max(0, g * C - i0)) : 0; };
        auto hi = [&](int g) { return tri == 2 ? max(0, min(R, (g + 1) * C - i0)) : R; };
        int n_items = 0;
        for (int g = 0; g < G; ++g) n_items += max(0, hi(g) - lo(g));
        for (int item = tid; item < n_items; item += nt) {
            int g = 0, base = 0;
            for (;; ++g) {
                const int n = max(0, hi(g) - lo(g));
                if (item < base + n) break;
                base += n;
            }
            const int r = lo(g) + item - base, i = i0 + r;
            int k0 = g * C;
            int k1 = min(K, k0 + C);
            if (tri == 1) k1 = min(k1, i + 1);
            if (tri == 2) k0 = max(k0, i);
            const double* a = A + i;
            double a0 = 0.0, a1 = 0.0, a2 = 0.0;
#pragma unroll 4
            for (int k = k0; k < k1; ++k) {
                const double x = a[(long)k * lda];
                a0 += x * v[k];
                a1 += x * v[ldv + k];
                a2 += x * v[2 * ldv + k];
            }
            red[g * GV_ROWS + r] = a0;
            red[RS + g * GV_ROWS + r] = a1;
            red[2 * RS + g * GV_ROWS + r] = a2;
        }
        __syncthreads();
        if (tid < R) {
            double t0 = 0.0, t1 = 0.0, t2 = 0.0;
            for (int q = 0; q < G; ++q) {
                if (tid < lo(q) || tid >= hi(q)) continue;
                t0 += red[q * GV_ROWS + tid];
                t1 += red[RS + q * GV_ROWS + tid];
                t2 += red[2 * RS + q * GV_ROWS + tid];
            }
            fin(i0 + tid, t0, t1, t2);
        }
        __syncthreads();
    }
}

// Fronts of at most PS_SMALL nodes take the warp path: one warp per front,
// warp-synchronous, sums in plain k order; larger fronts take the CTA path.  A
// front's path depends only on its own size, so its bits do not depend on what
// else shares its level.
constexpr int PS_SMALL = DC_PS_SMALL;
constexpr int PS_WARPS = DC_PS_WARPS;    // small fronts per CTA
constexpr int PS_LD = PS_SMALL + 1;       // shared-memory column stride of the warp path (no bank conflicts)

// Right-hand side of position t of a front: the children's update entries that
// add into t (pull list pp, children in order), then b_t for a pivot (bt not
// null); the three columns go to w[0], w[stride], w[2 stride].  The sums are
// those of a child-by-child scatter into zeroed storage, in the same order.
__device__ __forceinline__ void ps_gather(const PSolveDev& ps, const int* __restrict__ pp, int t,
                                          const d4* __restrict__ bt, double* __restrict__ w, int stride) {
    double x = 0.0, y = 0.0, z = 0.0;
    for (int e = pp[t]; e < pp[t + 1]; ++e) {
        const d4 a = ld_cg(ps.acc + ps.pull_idx[e]);
        x += a.x;
        y += a.y;
        z += a.z;
    }
    if (bt) {
        const d4 a = ld(bt);
        x += a.x;
        y += a.y;
        z += a.z;
    }
    w[0] = x;
    w[stride] = y;
    w[2 * stride] = z;
}

// The static blocks a front's forward sweep reads, fetched into L2 ahead of use.
__device__ __forceinline__ void ps_fwd_prefetch(const PSolveDev& ps, int s) {
    const int ns = ps.p[s] / 3, fs = ps.f[s] / 3;
    prefetch_l2(ps.xinv + ps.xoff[s], sizeof(double) * ns * ns);
    prefetch_l2(ps.panel + ps.poff[s], sizeof(double) * fs * ns);
}
__device__ __forceinline__ void ps_bwd_prefetch(const PSolveDev& ps, int s) {
    const int ns = ps.p[s] / 3, nu = ps.f[s] / 3 - ns;
    prefetch_l2(ps.pant + ps.toff[s], sizeof(double) * ns * nu);
    prefetch_l2(ps.xinvt + ps.xoff[s], sizeof(double) * ns * ns);
}

__device__ __forceinline__ void ps_fwd_cta(const PSolveDev& ps, int s, const d4* __restrict__ b,
                                           d4* __restrict__ y, double* __restrict__ smd) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int begin = ps.begin[s], ns = ps.p[s] / 3, fs = ps.f[s] / 3, nu = fs - ns;
    double* w = smd;                   // [3][fs]
    double* yv = w + 3 * fs;           // [3][ns]
    double* red = yv + 3 * ns;         // [3][GV_MAXG * GV_ROWS]
    const int* pp = ps.pull_ptr + ps.pull_off[s];
    for (int t = tid; t < fs; t += nt) ps_gather(ps, pp, t, t < ns ? b + begin + t : nullptr, w + t, fs);
    __syncthreads();
    const double* X = ps.xinv + ps.xoff[s];
    const double* Pn = ps.panel + ps.poff[s];
    cm_gemv3(X, ns, ns, ns, 1, w, fs, red, [&](int i, double t0, double t1, double t2) {
        yv[i] = t0;
        yv[ns + i] = t1;
        yv[2 * ns + i] = t2;
    });
    d4* acc = ps.acc + ps.aoff[s];
    cm_gemv3(Pn + ns, fs, nu, ns, 0, yv, ns, red, [&](int i, double t0, double t1, double t2) {
        st(acc + i, w[ns + i] - t0, w[fs + ns + i] - t1, w[2 * fs + ns + i] - t2);
    });
    for (int t = tid; t < ns; t += nt) st(y + begin + t, yv[t], yv[ns + t], yv[2 * ns + t]);
}

// Warp path, forward: w is this warp's [3][PS_LD] gathered right-hand side, then
// [3][PS_LD] of y_s.  Both products give one lane to each (row, column) pair, so
// that a front of ns or nu rows keeps 3 ns or 3 nu lanes busy instead of ns or
// nu (the fronts here have 4-24 pivot rows); a pair's sum runs over k in
// ascending order, as with one lane per row.
__device__ __forceinline__ void ps_fwd_warp(const PSolveDev& ps, int s, const d4* __restrict__ b,
                                            d4* __restrict__ y, double* __restrict__ w) {
    constexpr int L = PS_LD;
    const int lane = threadIdx.x & 31;
    const int begin = ps.begin[s], ns = ps.p[s] / 3, fs = ps.f[s] / 3, nu = fs - ns;
    double* yv = w + 3 * L;
    const int* pp = ps.pull_ptr + ps.pull_off[s];
    for (int t = lane; t < fs; t += 32) ps_gather(ps, pp, t, t < ns ? b + begin + t : nullptr, w + t, L);
    __syncwarp();
    // y_s = L_ss^-1 w_s (lower triangle)
    const double* X = ps.xinv + ps.xoff[s];
    for (int q = lane; q < 3 * ns; q += 32) {
        const int i = q / 3, col = q - 3 * i;
        const double* wc = w + col * L;
        double a = 0.0;
#pragma unroll 4
        for (int k = 0; k <= i; ++k) a += X[(long)k * ns + i] * wc[k];
        yv[col * L + i] = a;
    }
    __syncwarp();
    // update vector: w_U - L_Us y_s
    const double* Pn = ps.panel + ps.poff[s] + ns;
    double* acc = reinterpret_cast<double*>(ps.acc + ps.aoff[s]);
    for (int q = lane; q < 3 * nu; q += 32) {
        const int i = q / 3, col = q - 3 * i;
        const double* yc = yv + col * L;
        double a = 0.0;
#pragma unroll 4
        for (int k = 0; k < ns; ++k) a += Pn[(long)k * fs + i] * yc[k];
        acc[4 * i + col] = w[col * L + ns + i] - a;
    }
    for (int t = lane; t < ns; t += 32) st(y + begin + t, yv[t], yv[L + t], yv[2 * L + t]);
}

// Level kernel of L y = b: CTAs [0, n_big) take one large front each, the others
// PS_WARPS small fronts each (one per warp).
__global__ void __launch_bounds__(256) k_ps_fwd(PSolveDev ps, const int* __restrict__ big, int n_big,
                                                const int* __restrict__ small, int n_small,
                                                const d4* __restrict__ b, d4* __restrict__ y) {
    extern __shared__ double smd[];
    if ((int)blockIdx.x < n_big) {
        ps_fwd_prefetch(ps, big[blockIdx.x]);
        ps_fwd_cta(ps, big[blockIdx.x], b, y, smd);
        return;
    }
    const int warp = threadIdx.x >> 5;
    const int q = ((int)blockIdx.x - n_big) * PS_WARPS + warp;
    if (q < n_small) ps_fwd_warp(ps, small[q], b, y, smd + warp * 6 * PS_LD);
}

template <bool YL2 = false>
__device__ __forceinline__ void ps_bwd_cta(const PSolveDev& ps, const DevParams& P, int s, const d4* __restrict__ y,
                                           d4* __restrict__ out, int mode, const int* __restrict__ contact,
                                           const d4* __restrict__ nb, const double* __restrict__ cc,
                                           d4* __restrict__ f, int* __restrict__ case_, double* __restrict__ c_out,
                                           double* __restrict__ smd) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int begin = ps.begin[s], ns = ps.p[s] / 3, fs = ps.f[s] / 3, nu = fs - ns;
    double* w = smd;                   // [3][ns]
    double* xu = w + 3 * ns;           // [3][nu]
    double* red = xu + 3 * nu;         // [3][GV_MAXG * GV_ROWS]
    const int* un = ps.unode + ps.uptr[s];
    for (int t = tid; t < ns; t += nt) {
        const d4 a = YL2 ? ld_cg(y + begin + t) : ld(y + begin + t);   // y written in the same launch: L2 only
        w[t] = a.x;
        w[ns + t] = a.y;
        w[2 * ns + t] = a.z;
    }
    for (int k = tid; k < nu; k += nt) {
        const d4 a = ld_cg(ps.xint + un[k]);
        xu[k] = a.x;
        xu[nu + k] = a.y;
        xu[2 * nu + k] = a.z;
    }
    __syncthreads();
    // w -= L_Us^T x_U (the transposed update block is ns x nu column-major)
    cm_gemv3(ps.pant + ps.toff[s], ns, ns, nu, 0, xu, nu, red, [&](int i, double t0, double t1, double t2) {
        w[i] -= t0;
        w[ns + i] -= t1;
        w[2 * ns + i] -= t2;
    });
    // x = L_ss^-T w, then the per-node output
    cm_gemv3(ps.xinvt + ps.xoff[s], ns, ns, ns, 2, w, ns, red, [&](int i, double t0, double t1, double t2) {
        const int row = begin + i;
        st(ps.xint + row, t0, t1, t2);
        finish_row(P, row, t0, t1, t2, out, mode, contact, nb, cc, f, case_, c_out);
    });
}

// Warp path, backward: w is this warp's [3][PS_LD] right-hand side, then
// [3][PS_LD] of x_U, later of x_s.  One lane per (row, column) pair, as forward.
template <bool YL2 = false>
__device__ __forceinline__ void ps_bwd_warp(const PSolveDev& ps, const DevParams& P, int s, const d4* __restrict__ y,
                                            d4* __restrict__ out, int mode, const int* __restrict__ contact,
                                            const d4* __restrict__ nb, const double* __restrict__ cc,
                                            d4* __restrict__ f, int* __restrict__ case_,
                                            double* __restrict__ c_out, double* __restrict__ w) {
    constexpr int L = PS_LD;
    const int lane = threadIdx.x & 31;
    const int begin = ps.begin[s], ns = ps.p[s] / 3, fs = ps.f[s] / 3, nu = fs - ns;
    double* xu = w + 3 * L;
    const int* un = ps.unode + ps.uptr[s];
    for (int t = lane; t < ns; t += 32) {
        const d4 a = YL2 ? ld_cg(y + begin + t) : ld(y + begin + t);
        w[t] = a.x;
        w[L + t] = a.y;
        w[2 * L + t] = a.z;
    }
    for (int k = lane; k < nu; k += 32) {
        const d4 a = ld_cg(ps.xint + un[k]);
        xu[k] = a.x;
        xu[L + k] = a.y;
        xu[2 * L + k] = a.z;
    }
    __syncwarp();
    // w_s -= L_Us^T x_U (the transposed update block is ns x nu column-major)
    const double* T = ps.pant + ps.toff[s];
    for (int q = lane; q < 3 * ns; q += 32) {
        const int i = q / 3, col = q - 3 * i;
        const double* xc = xu + col * L;
        double a = 0.0;
#pragma unroll 4
        for (int k = 0; k < nu; ++k) a += T[(long)k * ns + i] * xc[k];
        w[col * L + i] -= a;
    }
    __syncwarp();
    // x_s = L_ss^-T w_s (upper triangle of the transposed inverse), into xu
    const double* XT = ps.xinvt + ps.xoff[s];
    for (int q = lane; q < 3 * ns; q += 32) {
        const int i = q / 3, col = q - 3 * i;
        const double* wc = w + col * L;
        double a = 0.0;
#pragma unroll 4
        for (int k = i; k < ns; ++k) a += XT[(long)k * ns + i] * wc[k];
        xu[col * L + i] = a;
    }
    __syncwarp();
    for (int t = lane; t < ns; t += 32) {
        const double a0 = xu[t], a1 = xu[L + t], a2 = xu[2 * L + t];
        const int row = begin + t;
        st(ps.xint + row, a0, a1, a2);
        finish_row(P, row, a0, a1, a2, out, mode, contact, nb, cc, f, case_, c_out);
    }
}

// Level kernel of L^T x = y (and the per-node output): large fronts per CTA, small
// fronts per warp, as for the forward sweep.
__global__ void __launch_bounds__(256) k_ps_bwd(PSolveDev ps, DevParams P, const int* __restrict__ big, int n_big,
                                                const int* __restrict__ small, int n_small, const d4* __restrict__ y,
                                                d4* __restrict__ out, int mode, const int* __restrict__ contact,
                                                const d4* __restrict__ nb, const double* __restrict__ cc,
                                                d4* __restrict__ f, int* __restrict__ case_,
                                                double* __restrict__ c_out) {
    extern __shared__ double smd[];
    if ((int)blockIdx.x < n_big) {
        ps_bwd_prefetch(ps, big[blockIdx.x]);
        ps_bwd_cta(ps, P, big[blockIdx.x], y, out, mode, contact, nb, cc, f, case_, c_out, smd);
        return;
    }
    const int warp = threadIdx.x >> 5;
    const int q = ((int)blockIdx.x - n_big) * PS_WARPS + warp;
    if (q < n_small)
        ps_bwd_warp(ps, P, small[q], y, out, mode, contact, nb, cc, f, case_, c_out, smd + warp * 6 * PS_LD);
}

// ---- tree-scheduled sweeps: one launch per sweep instead of one per level.
// CTAs take work items from a ticket counter in a topological order (children
// before parents for L y = b, the reverse for L^T x = y) and, before an item,
// wait for the done flags of the fronts it reads: its children's update vectors
// (forward) or its parent's solution (backward; the parent's own wait covers the
// ancestors above it).  An item only waits on items with smaller tickets, which
// CTAs already running hold, and the smallest unfinished ticket never waits, so
// the launch makes progress whatever the number of CTAs resident.  A front's
// arithmetic is that of the level kernels, so the results are the same bits.
// Every wait is bounded (dc_wait.cuh): one that gives up sets the sticky fault
// word, and every CTA stops taking items once the word is set.

// One thread takes the next ticket for the CTA; n_items once the fault word is set.
__device__ __forceinline__ int ps_take(const PSolveDev& ps, int* ticket, int* s_item) {
    if (threadIdx.x == 0) *s_item = dc_fault_set(ps.fault) ? ps.n_items : atomicAdd(ticket, 1);
    __syncthreads();
    return *s_item;
}

__global__ void __launch_bounds__(256) k_ps_fwd_tree(PSolveDev ps, const d4* __restrict__ b, d4* __restrict__ y) {
    extern __shared__ double smd[];
    __shared__ int s_item, s_ok;
    int* ticket = ps.sched;
    int* done = ps.sched + 1;
    for (;;) {
        const int it = ps_take(ps, ticket, &s_item);
        if (it >= ps.n_items) return;
        const int q0 = ps.tq_ptr[it], nq = ps.tq_ptr[it + 1] - q0;
        const int s0 = ps.tq_sn[q0];
        if (ps.f[s0] / 3 > PS_SMALL) {
            ps_fwd_prefetch(ps, s0);
            if (threadIdx.x == 0) {
                bool ok = true;
                for (int q = ps.cptr[s0]; ok && q < ps.cptr[s0 + 1]; ++q) ok = dc_wait_flag(done + ps.child[q], ps.fault);
                s_ok = ok;
            }
            __syncthreads();
            if (!s_ok) return;
            ps_fwd_cta(ps, s0, b, y, smd);
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) dc_st_release(done + s0, 1);
        } else {
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            if (warp < nq) {
                const int s = ps.tq_sn[q0 + warp];
                int ok = 1;
                if (lane == 0)
                    for (int q = ps.cptr[s]; ok && q < ps.cptr[s + 1]; ++q) ok = dc_wait_flag(done + ps.child[q], ps.fault);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (ok) {
                    ps_fwd_warp(ps, s, b, y, smd + warp * 6 * PS_LD);
                    __threadfence();
                    __syncwarp();
                    if (lane == 0) dc_st_release(done + s, 1);
                }
            }
            __syncthreads();   // every warp has read s_item before it is rewritten
        }
    }
}

__global__ void __launch_bounds__(256) k_ps_bwd_tree(PSolveDev ps, DevParams P, const d4* __restrict__ y,
                                                     d4* __restrict__ out, int mode, const int* __restrict__ contact,
                                                     const d4* __restrict__ nb, const double* __restrict__ cc,
                                                     d4* __restrict__ f, int* __restrict__ case_,
                                                     double* __restrict__ c_out) {
    extern __shared__ double smd[];
    __shared__ int s_item, s_ok;
    int* ticket = ps.sched + ps.S + 1;
    int* done = ps.sched + ps.S + 2;
    for (;;) {
        const int t = ps_take(ps, ticket, &s_item);
        if (t >= ps.n_items) return;
        const int it = ps.n_items - 1 - t;   // the forward order reversed: parents first
        const int q0 = ps.tq_ptr[it], nq = ps.tq_ptr[it + 1] - q0;
        const int s0 = ps.tq_sn[q0];
        if (ps.f[s0] / 3 > PS_SMALL) {
            ps_bwd_prefetch(ps, s0);
            if (threadIdx.x == 0) {
                const int par = ps.parent[s0];
                s_ok = par < 0 || dc_wait_flag(done + par, ps.fault);
            }
            __syncthreads();
            if (!s_ok) return;
            ps_bwd_cta(ps, P, s0, y, out, mode, contact, nb, cc, f, case_, c_out, smd);
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) dc_st_release(done + s0, 1);
        } else {
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            if (warp < nq) {
                const int s = ps.tq_sn[q0 + warp];
                int ok = 1;
                if (lane == 0) {
                    const int par = ps.parent[s];
                    ok = par < 0 || dc_wait_flag(done + par, ps.fault);
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (ok) {
                    ps_bwd_warp(ps, P, s, y, out, mode, contact, nb, cc, f, case_, c_out,
                                smd + warp * 6 * PS_LD);
                    __threadfence();
                    __syncwarp();
                    if (lane == 0) dc_st_release(done + s, 1);
                }
            }
            __syncthreads();
        }
    }
}

// Both sweeps of one global step as one launch: tickets [0, n) are the forward
// items, [n, 2n) the backward items (the forward order reversed).  A backward
// item waits for its parent's backward flag, or, at a root, for the root's
// forward flag; every wait is again on a smaller ticket, so the launch makes
// progress whatever the number of resident CTAs.  The backward work of small
// trees runs while the forward sweeps of large ones are still in their upper
// levels.  Same arithmetic as the two launches, so the same bits.
__global__ void __launch_bounds__(256) k_ps_sweeps_tree(PSolveDev ps, DevParams P, const d4* __restrict__ b,
                                                        d4* __restrict__ y, d4* __restrict__ out, int mode,
                                                        const int* __restrict__ contact,
                                                        const d4* __restrict__ nb, const double* __restrict__ cc,
                                                        d4* __restrict__ f, int* __restrict__ case_,
                                                        double* __restrict__ c_out) {
    extern __shared__ double smd[];
    __shared__ int s_item, s_ok;
    int* ticket = ps.sched;
    int* done_f = ps.sched + 1;
    int* done_b = ps.sched + ps.S + 2;
    const int n = ps.n_items;
    for (;;) {
        if (threadIdx.x == 0) s_item = dc_fault_set(ps.fault) ? 2 * n : atomicAdd(ticket, 1);
        __syncthreads();
        const int t = s_item;
        if (t >= 2 * n) return;
        const bool fwd = t < n;
        const int it = fwd ? t : n - 1 - (t - n);
        const int q0 = ps.tq_ptr[it], nq = ps.tq_ptr[it + 1] - q0;
        const int s0 = ps.tq_sn[q0];
        if (ps.f[s0] / 3 > PS_SMALL) {
            if (fwd) ps_fwd_prefetch(ps, s0);
            else ps_bwd_prefetch(ps, s0);
            if (threadIdx.x == 0) {
                bool ok = true;
                if (fwd) {
                    for (int q = ps.cptr[s0]; ok && q < ps.cptr[s0 + 1]; ++q)
                        ok = dc_wait_flag(done_f + ps.child[q], ps.fault);
                } else {
                    const int par = ps.parent[s0];
                    ok = par < 0 ? dc_wait_flag(done_f + s0, ps.fault) : dc_wait_flag(done_b + par, ps.fault);
                }
                s_ok = ok;
            }
            __syncthreads();
            if (!s_ok) return;
            if (fwd) ps_fwd_cta(ps, s0, b, y, smd);
            else ps_bwd_cta<true>(ps, P, s0, y, out, mode, contact, nb, cc, f, case_, c_out, smd);
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) dc_st_release((fwd ? done_f : done_b) + s0, 1);
        } else {
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            if (warp < nq) {
                const int s = ps.tq_sn[q0 + warp];
                int ok = 1;
                if (lane == 0) {
                    if (fwd) {
                        for (int q = ps.cptr[s]; ok && q < ps.cptr[s + 1]; ++q)
                            ok = dc_wait_flag(done_f + ps.child[q], ps.fault);
                    } else {
                        const int par = ps.parent[s];
                        ok = par < 0 ? dc_wait_flag(done_f + s, ps.fault) : dc_wait_flag(done_b + par, ps.fault);
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (ok) {
                    if (fwd) ps_fwd_warp(ps, s, b, y, smd + warp * 6 * PS_LD);
                    else ps_bwd_warp<true>(ps, P, s, y, out, mode, contact, nb, cc, f, case_, c_out,
                                           smd + warp * 6 * PS_LD);
                    __threadfence();
                    __syncwarp();
                    if (lane == 0) dc_st_release((fwd ? done_f : done_b) + s, 1);
                }
            }
            __syncthreads();   // every warp has read s_item before it is rewritten
        }
    }
}

__global__ void k_finalize(int m, double h, const d4* __restrict__ x_n, const d4* __restrict__ v,
                           d4* __restrict__ x1, unsigned long long* __restrict__ nonfinite) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    d4 a = ld(x_n + i), b = ld(v + i);
    const double x = a.x + h * b.x, y = a.y + h * b.y, z = a.z + h * b.z;
    st(x1 + i, x, y, z);
    if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(b.x) && isfinite(b.y) && isfinite(b.z)))
        atomicExch(nonfinite, 1ull);
}

// Instances that have taken their own number of steps keep their state.
__global__ void k_freeze(int m, int m_free, const int* __restrict__ node_inst, const int* __restrict__ inst_steps,
                         int step, const int* __restrict__ step_base, const d4* __restrict__ xin,
                         const d4* __restrict__ vin, d4* __restrict__ xout, d4* __restrict__ vout,
                         int* __restrict__ contact) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m || inst_steps[node_inst[i]] > step + (step_base ? *step_base : 0)) return;
    const d4 x = ld(xin + i), v = ld(vin + i);
    st(xout + i, x.x, x.y, x.z);
    st(vout + i, v.x, v.y, v.z);
    if (i < m_free) contact[i] = -1;
}

__global__ void k_set_int(int* p, int v) { *p = v; }

__global__ void k_pass_adjoint(int m, const int* __restrict__ node_inst, const int* __restrict__ inst_steps,
                               int step, const d4* __restrict__ gv_in, d4* __restrict__ gv_out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m || inst_steps[node_inst[i]] > step) return;
    const d4 g = ld(gv_in + i);
    st(gv_out + i, g.x, g.y, g.z);
}

// Global step of the mass splitting (Eq. ly_et_al_govrningEq as printed):
// v_half = M^-1 b per free node, then the node's contact update.
__global__ void k_mass_solve(DevMesh dm, DevParams P, const d4* __restrict__ b, d4* __restrict__ v,
                             const int* __restrict__ contact, const d4* __restrict__ nb,
                             const double* __restrict__ cc, d4* __restrict__ f, int* __restrict__ case_) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dm.m_free) return;
    const d4 q = ld(b + i);
    const double mi = dm.mass[i];
    finish_row(P, i, q.x / mi, q.y / mi, q.z / mi, v, 1, contact, nb, cc, f, case_, nullptr);
}

__global__ void k_count_cases(const int* __restrict__ contact, const int* __restrict__ case_, int n,
                              unsigned long long* counters) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || contact[i] < 0) return;
    atomicAdd(counters + case_[i], 1ull);
}

inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

void launch_permute_in(const double* ext, d4* out, const int* int2ext, int m, int layout, cudaStream_t s) {
    dc_note_launch();
    const bool cm = layout == DC_LAYOUT_COMPONENT_MAJOR;
    k_permute_in<<<nblk(m, 256), 256, 0, s>>>(ext, out, int2ext, m, cm ? 1 : 3, cm ? (long)m : 1L);
}
void launch_permute_out(const d4* in, double* ext, const int* int2ext, int m, int layout, cudaStream_t s) {
    dc_note_launch();
    const bool cm = layout == DC_LAYOUT_COMPONENT_MAJOR;
    k_permute_out<<<nblk(m, 256), 256, 0, s>>>(in, ext, int2ext, m, cm ? 1 : 3, cm ? (long)m : 1L);
}
void launch_zero_pins(d4* v, int m_free, int m, cudaStream_t s) {
    if (m > m_free) {
        dc_note_launch();
        k_zero_range<<<nblk(m - m_free, 256), 256, 0, s>>>(v, m_free, m);
    }
}
void launch_detect(const DevMesh& dm, const DevParams& P, const d4* x_n, const d4* v_n, int* contact,
                   d4* nb, d4* f, d4* ind, cudaStream_t s) {
    dc_note_launch();
    k_detect<<<nblk(dm.m_free, dm.bs_node), dm.bs_node, 0, s>>>(dm, P, x_n, v_n, contact, nb, f, ind);
}
void launch_local(const DevMesh& dm, const DevParams& P, const d4* x_n, const d4* v, d4* c1, d4* c2,
                  d4* bu, cudaStream_t s) {
    dc_note_launch();
    k_local<<<nblk((long)dm.T + dm.m, dm.bs_local), dm.bs_local, 0, s>>>(dm, P, x_n, v, c1, c2, bu);
}
void launch_gather_rhs(const DevMesh& dm, const DevParams& P, const d4* v_n, const d4* c1, const d4* c2,
                       const d4* bu, const d4* f, d4* b, cudaStream_t s) {
    dc_note_launch();
    k_gather_rhs<<<nblk(dm.m_free, dm.bs_gather), dm.bs_gather, 0, s>>>(dm, P, v_n, c1, c2, bu, f, b);
}
namespace {
size_t ps_smem(int fs) { return (6 * (size_t)fs + 3 * (size_t)GV_ROWS * GV_MAXG) * sizeof(double); }
// CTA-path fronts get 128 threads up to 96 nodes, else 256; the warp path needs 256
int ps_threads(int big_fs, int n_small) { return (n_small > 0 || big_fs > 96) ? 256 : 128; }
size_t ps_level_smem(int big_fs, int n_small) {
    const size_t a = big_fs > 0 ? ps_smem(big_fs) : 0;
    const size_t b = n_small > 0 ? (size_t)PS_WARPS * 6 * PS_LD * sizeof(double) : 0;
    return a > b ? a : b;
}
}  // namespace

// The level kernels' dynamic shared-memory limit is shared by every context of
// the process: it only ever grows.
cudaError_t psolve_configure(int max_fs) {
    static std::mutex mu;
    static size_t configured = 48 * 1024;
    std::lock_guard<std::mutex> lock(mu);
    const size_t need = ps_level_smem(max_fs, 1);
    if (need <= configured) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_ps_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ps_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ps_fwd_tree, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ps_bwd_tree, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ps_sweeps_tree, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    if (e == cudaSuccess) configured = need;
    return e;
}

cudaError_t psolve_tree_grid(int max_fs, int* grid_f, int* grid_b, size_t* smem_out) {
    const size_t smem = ps_level_smem(max_fs, 1);
    *smem_out = smem;
    int dev = 0, sms = 0, nf = 0, nb = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nf, k_ps_fwd_tree, 256, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ps_bwd_tree, 256, smem);
    if (e != cudaSuccess) return e;
    *grid_f = sms * std::max(1, nf);
    *grid_b = sms * std::max(1, nb);
    return cudaSuccess;
}

void launch_solve_fwd(const DevMesh& dm, const d4* b, d4* y, cudaStream_t s) {
    if (dm.solver == 1) {
        const PSolveDev& ps = dm.ps;
        if (ps.tree) {
            if (ps.n_items == 0) return;
            cudaMemsetAsync(ps.sched, 0, sizeof(int) * (ps.S + 1), s);
            dc_note_launch();
            k_ps_fwd_tree<<<std::min(ps.tree_grid_f, ps.n_items), 256, ps.tree_smem, s>>>(ps, b, y);
            return;
        }
        for (int l = 0; l < ps.nlev; ++l) {
            const int nb = ps.nbig_h[l], nsm = ps.nsmall_h[l];
            if (nb + nsm <= 0) continue;
            const int* big = ps.sn + ps.lvl_ptr_h[l];
            const int grid = nb + (nsm + PS_WARPS - 1) / PS_WARPS;
            dc_note_launch();
            k_ps_fwd<<<grid, ps_threads(ps.maxbig_h[l], nsm), ps_level_smem(ps.maxbig_h[l], nsm), s>>>(
                ps, big, nb, big + nb, nsm, b, y);
        }
        return;
    }
    dc_note_launch();
    k_solve_fwd<<<dm.n_long + nblk(dm.n_short, 8), 256, 0, s>>>(dm, b, y);
}
void launch_solve_fwd_skip(const DevMesh& dm, const d4* b, d4* y, int skip, cudaStream_t s) {
    const PSolveDev& ps = dm.ps;
    cudaMemsetAsync(ps.sched, 0, sizeof(int) * (ps.S + 1), s);
    const int ticket = skip;   // pageable source: copied before the call returns
    cudaMemcpyAsync(ps.sched, &ticket, sizeof(int), cudaMemcpyHostToDevice, s);
    dc_note_launch();
    k_ps_fwd_tree<<<std::min(ps.tree_grid_f, ps.n_items), 256, ps.tree_smem, s>>>(ps, b, y);
}
void launch_solve_bwd(const DevMesh& dm, const DevParams& P, const d4* y, d4* out, int mode, const int* contact,
                      const d4* nb, const double* c, d4* f, int* case_, double* c_out, cudaStream_t s) {
    if (dm.solver == 1) {
        const PSolveDev& ps = dm.ps;
        if (ps.tree) {
            if (ps.n_items == 0) return;
            cudaMemsetAsync(ps.sched + ps.S + 1, 0, sizeof(int) * (ps.S + 1), s);
            dc_note_launch();
            k_ps_bwd_tree<<<std::min(ps.tree_grid_b, ps.n_items), 256, ps.tree_smem, s>>>(
                ps, P, y, out, mode, contact, nb, c, f, case_, c_out);
            return;
        }
        for (int l = ps.nlev - 1; l >= 0; --l) {
            const int nbg = ps.nbig_h[l], nsm = ps.nsmall_h[l];
            if (nbg + nsm <= 0) continue;
            const int* big = ps.sn + ps.lvl_ptr_h[l];
            const int grid = nbg + (nsm + PS_WARPS - 1) / PS_WARPS;
            dc_note_launch();
            k_ps_bwd<<<grid, ps_threads(ps.maxbig_h[l], nsm), ps_level_smem(ps.maxbig_h[l], nsm), s>>>(
                ps, P, big, nbg, big + nbg, nsm, y, out, mode, contact, nb, c, f, case_, c_out);
        }
        return;
    }
    dc_note_launch();
    k_solve_bwd<<<nblk((long)dm.m_free * 32, 256), 256, 0, s>>>(dm, P, y, out, mode, contact, nb, c, f, case_,
                                                                c_out);
}
bool launch_solve_sweeps(const DevMesh& dm, const DevParams& P, const d4* b, d4* y, d4* out, int mode,
                         const int* contact, const d4* nb, const double* c, d4* f, int* case_, double* c_out,
                         cudaStream_t s) {
    const PSolveDev& ps = dm.ps;
    if (dm.solver != 1 || !ps.tree || !ps.fused) return false;
    if (ps.n_items == 0) return true;
    cudaMemsetAsync(ps.sched, 0, sizeof(int) * 2 * (ps.S + 1), s);
    dc_note_launch();
    k_ps_sweeps_tree<<<std::min(std::max(ps.tree_grid_f, ps.tree_grid_b), 2 * ps.n_items), 256, ps.tree_smem, s>>>(
        ps, P, b, y, out, mode, contact, nb, c, f, case_, c_out);
    return true;
}
void launch_finalize(const DevMesh& dm, const DevParams& P, const d4* x_n, const d4* v, d4* x_np1,
                     unsigned long long* nonfinite, cudaStream_t s) {
    dc_note_launch();
    k_finalize<<<nblk(dm.m, dm.bs_node), dm.bs_node, 0, s>>>(dm.m, P.h, x_n, v, x_np1, nonfinite);
}
void launch_freeze(const DevMesh& dm, const DevParams& P, const int* inst_steps, int step, const int* step_base,
                   const d4* xin, const d4* vin, d4* xout, d4* vout, int* contact, cudaStream_t s) {
    dc_note_launch();
    k_freeze<<<nblk(dm.m, 256), 256, 0, s>>>(dm.m, dm.m_free, P.node_inst, inst_steps, step, step_base, xin, vin,
                                             xout, vout, contact);
}
void launch_set_int(int* p, int v, cudaStream_t s) {
    dc_note_launch();
    k_set_int<<<1, 1, 0, s>>>(p, v);
}
void launch_pass_adjoint(const DevMesh& dm, const DevParams& P, const int* inst_steps, int step, const d4* gv_in,
                         d4* gv_out, cudaStream_t s) {
    dc_note_launch();
    k_pass_adjoint<<<nblk(dm.m, 256), 256, 0, s>>>(dm.m, P.node_inst, inst_steps, step, gv_in, gv_out);
}
void launch_mass_solve(const DevMesh& dm, const DevParams& P, const d4* b, d4* v, const int* contact, const d4* nb,
                       const double* c, d4* f, int* case_, cudaStream_t s) {
    dc_note_launch();
    k_mass_solve<<<nblk(dm.m_free, dm.bs_node), dm.bs_node, 0, s>>>(dm, P, b, v, contact, nb, c, f, case_);
}
void launch_count_cases(const int* contact, const int* case_, int m_free, unsigned long long* counters,
                        cudaStream_t s) {
    dc_note_launch();
    k_count_cases<<<nblk(m_free, 256), 256, 0, s>>>(contact, case_, m_free, counters);
}
