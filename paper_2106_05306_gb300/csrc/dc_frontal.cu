// Per-step single-precision multifrontal LDL^T of the constrained adjoint
// matrix, used as the preconditioner of the FP64 adjoint Krylov solve.
//
// The matrix factorised is H^ = T H T + (I - T T) with H = P - Delta P - Delta R
// (Sec. 4, Eq. ppr_adjoint) and a per-node T: the identity for free nodes, 0 for
// stick nodes, the tangent-plane projector I - n n^T for slip nodes.  It differs
// from the exact constrained operator only by the obliqueness of the slip
// constraint and by single-precision rounding; the outer FP64 GMRES removes both.
// No pivoting beyond the supernode order; a pivot below tau is replaced by
// +-tau (the preconditioner stays usable, GMRES corrects).
//
// Fronts are dense column-major f x f blocks (DOF granularity, 3 per node) in
// one pool; only their lower triangles are used.  One CTA handles one front; on
// levels of larger fronts the rank-32 trailing updates run on the tensor cores
// (tcgen05, TF32 split in three passes, see tc_trailing_update).
#include <mutex>

#include "dc_adjoint.h"
#include "dc_internal.h"
#include "dc_tc.cuh"
#include "dc_wait.cuh"

namespace {

constexpr int PB = 32;        // panel width of the blocked factorisation
constexpr int LDS = PB + 1;   // shared-memory row stride (no bank conflicts)
constexpr int FT = 1024;      // threads per solve CTA
constexpr int FT2 = 512;      // threads per factorisation CTA
constexpr int TM = 8;         // register tile of the trailing update
// Tensor-core trailing update: 128 x TC_N accumulator tiles in TMEM, operands in
// shared memory (A: 128 rows, B: TC_N rows, each as TF32 hi and lo parts).
constexpr int TC_M = 128;
constexpr int TC_N = 64;
constexpr uint32_t TC_COLS = 64;                          // TMEM columns per CTA
constexpr int TC_A_BYTES = TC_M * TC_K * 4;               // one part of A
constexpr int TC_B_BYTES = TC_N * TC_K * 4;               // one part of B
constexpr int TC_FLOATS = (2 * TC_A_BYTES + 2 * TC_B_BYTES) / 4;
constexpr int TC_MIN_N2 = 64;                             // smaller trailing blocks: FMA path
constexpr int TC_MIN_F = 160;                             // levels with smaller fronts: FMA path
constexpr int TC_WAIT = 1 << 22;                          // polls of an MMA completion

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

// Node transform of the constraint: 0 free, 1 stick, 2 slip (normal n).
__device__ __forceinline__ void node_T(int type, const double n[3], double T[9]) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double v = (r == c) ? 1.0 : 0.0;
            if (type == 1) v = 0.0;
            else if (type == 2) v -= n[r] * n[c];
            T[3 * r + c] = v;
        }
}

// One 3x3 block H^_ij of the constrained matrix, written into its front.
__global__ void k_pairs(DevMesh dm, AdjDev ad, FrontDev fd) {
    int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= fd.NP) return;
    const int i = fd.pr_i[id], j = fd.pr_j[id];
    const double h2 = ad.h * ad.h;
    double H[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = fd.pr_cptr[id]; k < fd.pr_cptr[id + 1]; ++k) {
        int code = fd.pr_code[k];
        if (code >= 0) {
            int t = code / 9, a = (code / 3) % 3, b = code % 3;
            d4 g = ld(dm.G + t);
            double ga0, ga1, gb0, gb1;
            if (a == 1) { ga0 = g.x; ga1 = g.y; } else if (a == 2) { ga0 = g.z; ga1 = g.w; }
            else { ga0 = -(g.x + g.z); ga1 = -(g.y + g.w); }
            if (b == 1) { gb0 = g.x; gb1 = g.y; } else if (b == 2) { gb0 = g.z; gb1 = g.w; }
            else { gb0 = -(g.x + g.z); gb1 = -(g.y + g.w); }
            const d4 A0 = ld(ad.tr0 + t), A1 = ld(ad.tr1 + t), A2 = ld(ad.tr2 + t);
            const double s00 = A0.w, s01 = A1.w, s11 = A2.x, itr = A2.y;
            // the triangle's a_a, a_b and projector P, formed once per triangle
            const d4 va = ld(ad.tav + 4 * (long)t + a), vb = ld(ad.tav + 4 * (long)t + b);
            const d4 pp = ld(ad.tav + 4 * (long)t + 3);
            const double aa[3] = {va.x, va.y, va.z}, ab[3] = {vb.x, vb.y, vb.z};
            const double P[9] = {pp.x, pp.y, pp.z, pp.y, pp.w, A2.z, pp.z, A2.z, A2.w};
            double w = h2 * dm.wt[t];
            double gg = ga0 * gb0 + ga1 * gb1;
            double gam = ga0 * gb0 * s00 + (ga0 * gb1 + ga1 * gb0) * s01 + ga1 * gb1 * s11;
            double trS = itr > 0.0 ? 1.0 / itr : 0.0;   // 0 for a collapsed triangle (a_a = a_b = 0)
            // block = w ((g_a.g_b) I - trS a_a a_b^T - gam P)
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) {
                    double dl = (r == c) ? 1.0 : 0.0;
                    H[3 * r + c] += w * (gg * dl - trS * aa[r] * ab[c] - gam * P[3 * r + c]);
                }
        } else {
            int b = -code - 1;
            d4 q = ld(ad.bq + b);
            double w = h2 * dm.wb[b] * fd.pr_coef[k];
            double qh[3] = {q.x, q.y, q.z};
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c)
                    H[3 * r + c] += w * (((r == c) ? (1.0 - q.w) : 0.0) + q.w * qh[r] * qh[c]);
        }
    }
    int ti = ad.type[i], tj = ad.type[j];
    if (i == j) {
        double mi = dm.mass[i];
        H[0] += mi; H[4] += mi; H[8] += mi;
        if (ti == 2) {
            d4 sl = ld(ad.slip + i), nb = ld(ad.nb + i);
            double th[3] = {sl.x, sl.y, sl.z}, n[3] = {nb.x, nb.y, nb.z};
            double bh[3] = {n[1] * th[2] - n[2] * th[1], n[2] * th[0] - n[0] * th[2], n[0] * th[1] - n[1] * th[0]};
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) H[3 * r + c] += sl.w * bh[r] * bh[c];
        }
    }
    double Hc[9];
    if (ti == 0 && tj == 0) {
        for (int q = 0; q < 9; ++q) Hc[q] = H[q];
    } else {
        double ni[3] = {0, 0, 0}, nj[3] = {0, 0, 0};
        if (ti == 2) { d4 nb = ld(ad.nb + i); ni[0] = nb.x; ni[1] = nb.y; ni[2] = nb.z; }
        if (tj == 2) { d4 nb = ld(ad.nb + j); nj[0] = nb.x; nj[1] = nb.y; nj[2] = nb.z; }
        double Ti[9], Tj[9], M1[9];
        node_T(ti, ni, Ti);
        node_T(tj, nj, Tj);
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double s = 0;
                for (int q = 0; q < 3; ++q) s += H[3 * r + q] * Tj[3 * q + c];
                M1[3 * r + c] = s;
            }
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double s = 0;
                for (int q = 0; q < 3; ++q) s += Ti[3 * r + q] * M1[3 * q + c];
                Hc[3 * r + c] = s;
            }
        if (i == j)   // + (I - T): identity on the constrained directions
            for (int q = 0; q < 9; ++q) Hc[q] += ((q % 4) == 0 ? 1.0 : 0.0) - Ti[q];
    }
    float* F = fd.pool + fd.pr_dst[id];
    const long ldf = fd.pr_ld[id];
    for (int c = 0; c < 3; ++c)
        for (int r = 0; r < 3; ++r) F[c * ldf + r] = (float)Hc[3 * r + c];
}

// Rows [g0, g0 + nrows) of the panel (column k of row g at Lt[k ldt + g]),
// times Dd[k] when Dd is given, split into TF32 hi/lo parts in the operand layout;
// rows at or beyond n2 and columns at or beyond kb are zero.
__device__ __forceinline__ void tc_stage(const float* __restrict__ Lt, int ldt, int g0, int nrows, int n2, int kb,
                                         const float* __restrict__ Dd, unsigned char* hi, unsigned char* lo) {
    for (int e = threadIdx.x; e < nrows * (TC_K / 4); e += blockDim.x) {
        const int r = e % nrows, k4 = e / nrows, g = g0 + r;
        float v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = 4 * k4 + j;
            v[j] = (g < n2 && k < kb) ? Lt[k * ldt + g] * (Dd ? Dd[k] : 1.0f) : 0.0f;
        }
        float4 h, l;
        tc_split(v[0], h.x, l.x);
        tc_split(v[1], h.y, l.y);
        tc_split(v[2], h.z, l.z);
        tc_split(v[3], h.w, l.w);
        *reinterpret_cast<float4*>(hi + tc_off(r, 4 * k4)) = h;
        *reinterpret_cast<float4*>(lo + tc_off(r, 4 * k4)) = l;
    }
}

// Trailing update T -= L D L^T of one panel on the tensor cores: for every
// 128 x TC_N tile (I, J) of the n2 x n2 trailing block that meets its lower
// triangle, stage L's rows of tile I (A) and L D's rows of tile J (B), issue the
// three TF32 passes (hi hi, hi lo, lo hi; K = 32 in four slices each) from one
// thread into TMEM, and subtract the accumulator from T's lower entries (thread
// = row, coalesced down a column).  T is column-major with leading dimension f.
// Returns false (fault word set) if an MMA did not complete within TC_WAIT polls.
__device__ bool tc_trailing_update(float* __restrict__ T, int f, int n2, int kb, const float* __restrict__ Lt,
                                   int ldt, const float* __restrict__ Dd, unsigned char* tcs, uint32_t tmem,
                                   uint64_t* bar, uint32_t& phase, unsigned long long* fault) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nwg = blockDim.x >> 7, wg = warp >> 2, lq = warp & 3;
    unsigned char* a_hi = tcs;
    unsigned char* a_lo = a_hi + TC_A_BYTES;
    unsigned char* b_hi = a_lo + TC_A_BYTES;
    unsigned char* b_lo = b_hi + TC_B_BYTES;
    constexpr uint32_t idesc = tc_idesc_tf32(TC_M, TC_N);
    const int nI = (n2 + TC_M - 1) / TC_M, nJall = (n2 + TC_N - 1) / TC_N;
    for (int I = 0; I < nI; ++I) {
        const int r0 = I * TC_M;
        const int nJ = min((r0 + TC_M - 1) / TC_N + 1, nJall);
        for (int J = 0; J < nJ; ++J) {
            const int q0 = J * TC_N;
            if (J == 0) tc_stage(Lt, ldt, r0, TC_M, n2, kb, nullptr, a_hi, a_lo);
            tc_stage(Lt, ldt, q0, TC_N, n2, kb, Dd, b_hi, b_lo);
            tc_fence_async_smem();
            tc_fence_before_sync();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after_sync();
                const uint32_t ah = tc_smem_u32(a_hi), al = tc_smem_u32(a_lo);
                const uint32_t bh = tc_smem_u32(b_hi), bl = tc_smem_u32(b_lo);
#pragma unroll
                for (int pass = 0; pass < 3; ++pass) {
                    const uint32_t a = pass == 2 ? al : ah, b = pass == 1 ? bl : bh;
#pragma unroll
                    for (int kk = 0; kk < TC_K / 8; ++kk)
                        tc_mma_tf32(tmem, tc_desc(a + kk * 2 * TC_CORE_K_BYTES), tc_desc(b + kk * 2 * TC_CORE_K_BYTES),
                                    idesc, (pass | kk) ? 1u : 0u);
                }
                tc_commit(bar);
            }
            // this thread's row; the current values of its first 16-column chunk are
            // loaded while the tensor core works
            const int r = r0 + 32 * lq + lane;
            float old[16];
            {
                const int c0 = q0 + 16 * wg;
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    old[c] = (wg < TC_N / 16 && r < n2 && c0 + c <= r) ? T[(long)(c0 + c) * f + r] : 0.0f;
            }
            const bool done = tc_mbar_wait(bar, phase, TC_WAIT);
            phase ^= 1u;
            if (__syncthreads_or(!done)) {
                if (tid == 0) atomicExch(fault, 1ull);
                tc_mbar_wait(bar, phase ^ 1u, TC_WAIT);   // let an MMA still in flight finish
                return false;
            }
            tc_fence_after_sync();
            for (int ch = wg; ch < TC_N / 16; ch += nwg) {
                float v[16];
                tc_ld16(tmem + ((uint32_t)(32 * lq) << 16) + 16u * ch, v);
                const int c0 = q0 + 16 * ch;
                if (ch != wg) {
#pragma unroll
                    for (int c = 0; c < 16; ++c) old[c] = (r < n2 && c0 + c <= r) ? T[(long)(c0 + c) * f + r] : 0.0f;
                }
                if (r < n2) {
#pragma unroll
                    for (int c = 0; c < 16; ++c)
                        if (c0 + c <= r) T[(long)(c0 + c) * f + r] = old[c] - v[c];
                }
            }
            tc_fence_before_sync();
            __syncthreads();
        }
    }
    return true;
}

// Extend-add of the children's update blocks, then the partial LDL^T of the
// front's pivot columns; the trailing lower triangle becomes the update block.
// Per panel of PB pivot columns: the panel's diagonal block is staged row-major
// and its rows below transposed and zero-padded (the only copy of them, so that
// shared memory grows with one panel width, not two); warp 0 factorises the
// diagonal block in registers (shuffles only) and inverts it; every thread then
// solves its rows below the block against that inverse, in place; the trailing
// matrix is updated with TM x TM register tiles whose operands come from the
// transposed rows (128-bit shared-memory loads).
// Levels whose fronts are too large for one CTA's shared memory pass gscr: then
// the transposed rows and the scratch of the pivot-block inverse live in gscr
// (gsz floats per CTA, 16-byte aligned, read through L1/L2) and shared memory
// holds only the diagonal block, its inverse and the pivots.  The arithmetic and
// its order are the same either way.
// With tc set, trailing blocks of at least TC_MIN_N2 rows are updated on the
// tensor cores (tc_trailing_update; its operand buffers lead the shared memory)
// and smaller ones by the FMA tiles.
__global__ void __launch_bounds__(FT2) k_front_level(FrontDev fd, int lvl_begin, int mf, float* __restrict__ gscr,
                                                     long gsz, int tc) {
    extern __shared__ __align__(1024) float sm[];
    __shared__ uint64_t tc_bar;
    __shared__ uint32_t tc_slot;
    const int s = fd.lvl_sn[lvl_begin + blockIdx.x];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    float* F = fd.pool + fd.off[s];
    const int f = fd.f[s], p = fd.p[s];
    const int ldt = (mf + 7) / 8 * 8;                // row stride of the transposed panel
    float* const base = tc ? sm + TC_FLOATS : sm;
    float* Db = base;                                // [PB][LDS] diagonal block, row-major
    float* Xs = Db + PB * LDS;                       // [PB][LDS] diagonal-block inverse
    float* Dd = Xs + PB * LDS;                       // [PB] pivots of the panel
    float* const scr = gscr ? gscr + (long)blockIdx.x * gsz : base;
    // [PB][ldt] rows below the block, 16-byte aligned
    float* Lt = gscr ? scr : base + (2 * PB * LDS + PB + 3) / 4 * 4;
    uint32_t tmem = 0, tc_phase = 0;
    bool tc_ok = tc != 0;
    if (tc) {
        if (tid == 0) {
            tc_mbar_init(&tc_bar, 1);
            tc_mbar_init_fence();
        }
        if (warp == 0) tc_alloc(&tc_slot, TC_COLS);
        tc_fence_before_sync();
        __syncthreads();
        tc_fence_after_sync();
        tmem = tc_slot;
    }
    for (int q = fd.cptr[s]; q < fd.cptr[s + 1]; ++q) {
        const int c = fd.child[q];
        const float* Fc = fd.pool + fd.off[c];
        const int fc = fd.f[c], pc = fd.p[c], nu = fc - pc;
        const int* map = fd.cmap + fd.uptr[c];
        for (int b = warp; b < nu; b += nw) {
            const int pb = 3 * map[b / 3] + b % 3;
            const float* src = Fc + (long)(pc + b) * fc + pc;
            float* dst = F + (long)pb * f;
            // four rows per lane per round: loads first, then stores
            for (int a0 = b + lane; a0 < nu; a0 += 128) {
                float val[4], old[4];
                int di[4];
#pragma unroll
                for (int q2 = 0; q2 < 4; ++q2) {
                    const int a = a0 + 32 * q2;
                    di[q2] = (a < nu) ? 3 * map[a / 3] + a % 3 : -1;
                    val[q2] = (a < nu) ? src[a] : 0.0f;
                }
#pragma unroll
                for (int q2 = 0; q2 < 4; ++q2) old[q2] = (di[q2] >= 0) ? dst[di[q2]] : 0.0f;
#pragma unroll
                for (int q2 = 0; q2 < 4; ++q2)
                    if (di[q2] >= 0) dst[di[q2]] = old[q2] + val[q2];
            }
        }
        __syncthreads();
    }
    const float tau = fd.tau[s];
    float* binv = fd.binv + fd.binv_off[s];
    for (int k0 = 0; k0 < p; k0 += PB) {
        const int kb = min(PB, p - k0);
        const int nr = f - k0;
        const int n2 = nr - kb;                          // rows below the diagonal block
        const int n2p = (n2 + TM - 1) / TM * TM;
        for (int c = warp; c < kb; c += nw) {
            const float* src = F + (long)(k0 + c) * f + k0;
            for (int r = lane; r < nr; r += 32) {
                const float v = src[r];
                if (r < kb) Db[r * LDS + c] = v;
                else Lt[c * ldt + r - kb] = v;
            }
            for (int r = n2 + lane; r < n2p; r += 32) Lt[c * ldt + r] = 0.0f;
        }
        __syncthreads();
        if (warp == 0) {
            // lane r holds row r of the diagonal block
            float row[PB];
#pragma unroll
            for (int j = 0; j < PB; ++j) row[j] = (lane < kb && j < kb) ? Db[lane * LDS + j] : 0.0f;
#pragma unroll
            for (int c = 0; c < PB; ++c) {
                if (c < kb) {
                    float d = __shfl_sync(0xffffffffu, row[c], c);
                    if (fabsf(d) < tau) d = (d < 0.0f) ? -tau : tau;
                    const float id = 1.0f / d;
                    const float a_rc = row[c];                  // = l_r d for lanes below c
#pragma unroll
                    for (int j = c + 1; j < PB; ++j) {
                        const float lj = __shfl_sync(0xffffffffu, row[c], j) * id;
                        if (lane > c && j <= lane) row[j] -= a_rc * lj;
                    }
                    if (lane > c) row[c] = a_rc * id;
                    if (lane == c) row[c] = d;
                }
            }
            // column `lane` of X = L_dd^-1: X[i][c] = -sum_{k=c}^{i-1} L[i][k] X[k][c]
            float xc[PB];
#pragma unroll
            for (int i = 0; i < PB; ++i) xc[i] = (i == lane) ? 1.0f : 0.0f;
#pragma unroll
            for (int i = 1; i < PB; ++i) {
                float acc = 0.0f;
#pragma unroll
                for (int k = 0; k < i; ++k) acc += __shfl_sync(0xffffffffu, row[k], i) * xc[k];
                if (i > lane) xc[i] = -acc;
            }
            if (lane < kb) {
                float dl = 0.0f;
#pragma unroll
                for (int j = 0; j < PB; ++j) {
                    if (j <= lane && j < kb) Db[lane * LDS + j] = row[j];
                    if (j == lane) dl = row[j];
                }
                Dd[lane] = dl;
            }
#pragma unroll
            for (int i = 0; i < PB; ++i) Xs[i * LDS + lane] = (lane < kb && i < kb) ? xc[i] : (i == lane ? 1.0f : 0.0f);
            float* Bi = binv + (long)(k0 / PB) * PB * PB;   // column-major PB x PB
#pragma unroll
            for (int i = 0; i < PB; ++i) Bi[lane * PB + i] = (lane < kb && i < kb) ? xc[i] : (i == lane ? 1.0f : 0.0f);
        }
        __syncthreads();
        // rows below the diagonal block: l_r = D^-1 L_dd^-1 a_r (one row per thread,
        // in place in the transposed rows)
        for (int r = tid; r < n2; r += nt) {
            float a[PB];
#pragma unroll
            for (int j = 0; j < PB; ++j) a[j] = (j < kb) ? Lt[j * ldt + r] : 0.0f;
#pragma unroll
            for (int c = 0; c < PB; ++c) {
                if (c < kb) {
                    float sum = 0.0f;
#pragma unroll
                    for (int j = 0; j <= c; ++j) sum += Xs[c * LDS + j] * a[j];
                    Lt[c * ldt + r] = sum / Dd[c];
                }
            }
        }
        __syncthreads();
        // the panel's columns back to the front (disjoint from what the trailing
        // update below reads and writes, so no barrier between the two)
        for (int c = warp; c < kb; c += nw) {
            float* dst = F + (long)(k0 + c) * f + k0;
            for (int r = c + lane; r < nr; r += 32) dst[r] = r < kb ? Db[r * LDS + c] : Lt[c * ldt + r - kb];
        }
        if (tc_ok && n2 >= TC_MIN_N2) {
            tc_ok = tc_trailing_update(F + (long)(k0 + kb) * f + k0 + kb, f, n2, kb, Lt, ldt, Dd,
                                       reinterpret_cast<unsigned char*>(sm), tmem, &tc_bar, tc_phase, fd.fault);
            if (!tc_ok) break;
            continue;
        }
        // trailing update in TM x 4 half-tiles of the TM x TM tiles of the lower
        // triangle; each thread prefetches its tile's current values before the FMA
        // loop so that the memory latency overlaps the arithmetic
        const int nT = n2p / TM;
        const long nunits = (long)nT * (nT + 1);               // two halves per tile
        for (long t2 = tid; t2 < nunits; t2 += nt) {
            const long t = t2 >> 1;
            const int half = (int)(t2 & 1);
            // triangular tile index; single-precision sqrt, then exact integer fix-up
            int ti = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
            while ((long)(ti + 1) * (ti + 2) / 2 <= t) ++ti;
            while ((long)ti * (ti + 1) / 2 > t) --ti;
            const int tj = (int)(t - (long)ti * (ti + 1) / 2);
            const int r0 = TM * ti, c0 = TM * tj + 4 * half;   // relative to the trailing start
            float old[TM][4], acc[TM][4];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int col = kb + c0 + v;
                const float* dst = F + (long)(k0 + min(col, nr - 1)) * f + k0 + kb;
#pragma unroll
                for (int u = 0; u < TM; ++u) {
                    const int row = kb + r0 + u;
                    old[u][v] = (col < nr && row < nr && row >= col) ? dst[r0 + u] : 0.0f;
                    acc[u][v] = 0.0f;
                }
            }
            for (int c = 0; c < kb; ++c) {
                const float dc = Dd[c];
                const float4* la = reinterpret_cast<const float4*>(Lt + c * ldt + r0);
                const float4 a0 = la[0], a1 = la[1];
                const float4 b0 = *reinterpret_cast<const float4*>(Lt + c * ldt + c0);
                const float a[TM] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bv[4] = {b0.x * dc, b0.y * dc, b0.z * dc, b0.w * dc};
#pragma unroll
                for (int u = 0; u < TM; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * bv[v];
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int col = kb + c0 + v;
                if (col >= nr) continue;
                float* dst = F + (long)(k0 + col) * f + k0 + kb;
#pragma unroll
                for (int u = 0; u < TM; ++u) {
                    const int row = kb + r0 + u;
                    if (row < nr && row >= col) dst[r0 + u] = old[u][v] - acc[u][v];
                }
            }
        }
        __syncthreads();
    }
    // Explicit inverse X = L_ss^-1 of the unit-lower pivot block, by block rows:
    // X_II = B_I (the stored diagonal-block inverse), X_IJ = -B_I sum_{K=J}^{I-1} L_IK X_KJ.
    // X is column-major p x p.  Per block row I the rows L[i0.., 0..i0) are staged in
    // shared memory, and per block column J the needed part of X as well.
    float* X = fd.linv + fd.linv_off[s];
    const int nb = (tc && !tc_ok) ? 0 : (p + PB - 1) / PB;   // (nothing more after an MMA timeout)
    for (int I = 0; I < nb; ++I) {
        const int i0 = I * PB, ib = min(PB, p - i0);
        const float* Bi = binv + (long)I * PB * PB;
        const int lr = i0 + 1;                         // odd row stride: no bank conflicts
        float* Lrow = scr;                             // [PB][lr]: L[i0 + r][k], k < i0
        float* Xc = Lrow + (long)PB * lr;              // [PB][lr]: X[k][32J + c], k < i0
        float* T = Xc + (long)PB * lr;                 // [PB][PB] partial sums of one J
        for (long e = tid; e < (long)ib * i0; e += nt) {
            const int r = (int)(e % ib), k = (int)(e / ib);
            Lrow[r * lr + k] = F[(long)k * f + i0 + r];
        }
        for (int J = 0; J <= I; ++J) {
            const int k1 = J * PB;
            if (J < I) {
                for (long e = tid; e < (long)PB * (i0 - k1); e += nt) {
                    const int k = k1 + (int)(e % (i0 - k1)), c = (int)(e / (i0 - k1));
                    Xc[c * lr + k] = X[(long)(k1 + c) * p + k];
                }
                __syncthreads();
                // T[r][c] = sum_{k=32J}^{i0-1} L[i0 + r][k] X[k][32J + c]
                for (int e = tid; e < PB * PB; e += nt) {
                    const int r = e % PB, c = e / PB;
                    float acc = 0.0f;
                    if (r < ib) {
                        const float* lrow = Lrow + r * lr;
                        const float* xcol = Xc + c * lr;
#pragma unroll 8
                        for (int k = k1; k < i0; ++k) acc += lrow[k] * xcol[k];
                    }
                    T[c * PB + r] = acc;
                }
                __syncthreads();
            }
            // X_IJ[r][c] = -sum_q B_I[r][q] T[q][c]; X_II = B_I
            for (int e = tid; e < PB * PB; e += nt) {
                const int r = e % PB, c = e / PB;
                const int row = i0 + r, col = k1 + c;
                if (r >= ib || col >= p) continue;
                float v;
                if (J == I) {
                    v = Bi[c * PB + r];
                } else {
                    v = 0.0f;
                    for (int q = 0; q < ib; ++q) v -= Bi[q * PB + r] * T[c * PB + q];
                }
                X[(long)col * p + row] = v;
            }
            __syncthreads();
        }
        for (long e = tid; e < (long)ib * (p - i0); e += nt) {   // upper part of block row I: zero
            const int r = (int)(e % ib), col = i0 + (int)(e / ib);
            if (col > i0 + r) X[(long)col * p + i0 + r] = 0.0f;
        }
        __syncthreads();
    }
    if (tc) {
        tc_fence_before_sync();
        __syncthreads();
        tc_fence_after_sync();
        if (warp == 0) tc_dealloc(tmem, TC_COLS);
    }
}

// Issues L2 prefetches for [p, p + bytes) (128-byte lines, spread over the CTA),
// so that a front's blocks stream in from HBM while the CTA gathers its inputs.
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
    const char* c = static_cast<const char*>(p);
    for (size_t o = (size_t)threadIdx.x * 128; o < bytes; o += (size_t)blockDim.x * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(c + o));
}

// Column-major matrix-vector product on one CTA: t_i = sum_k A[k * lda + i] v_k for
// rows i < nrows and k < K (k <= i when tri).  Rows go in passes of GV_ROWS; the
// k range is cut into G contiguous chunks with G a function of K alone, every
// (row, chunk) partial sum is one work item (consecutive items take consecutive
// rows: coalesced), and a row's partial sums are added in chunk order.  The
// arithmetic thus depends only on (nrows, K), never on the CTA size, so a front
// gives the same bits whatever else shares its level.  fin(i, t_i) stores.
constexpr int GV_ROWS = 128;
constexpr int GV_MAXG = 8;
__host__ __device__ constexpr int gv_groups(int K) { return K <= 8 ? 1 : (K + 7) / 8 < GV_MAXG ? (K + 7) / 8 : GV_MAXG; }

template <class Fin>
__device__ __forceinline__ void cm_gemv(const float* __restrict__ A, long lda, int nrows, int K, bool tri,
                                        const float* __restrict__ v, float* __restrict__ red, Fin fin) {
    const int nt = blockDim.x, tid = threadIdx.x;
    const int G = gv_groups(K);
    const int C = (K + G - 1) / G;
    for (int i0 = 0; i0 < nrows; i0 += GV_ROWS) {
        for (int item = tid; item < GV_ROWS * G; item += nt) {
            const int r = item % GV_ROWS, g = item / GV_ROWS, i = i0 + r;
            float acc = 0.0f;
            if (i < nrows) {
                const int k0 = g * C;
                int k1 = min(K, k0 + C);
                if (tri) k1 = min(k1, i + 1);
                const float* a = A + i;
#pragma unroll 4
                for (int k = k0; k < k1; ++k) acc += a[(long)k * lda] * v[k];
            }
            red[g * GV_ROWS + r] = acc;
        }
        __syncthreads();
        if (tid < GV_ROWS && i0 + tid < nrows) {
            float t = 0.0f;
            for (int q = 0; q < G; ++q) t += red[q * GV_ROWS + tid];
            fin(i0 + tid, t);
        }
        __syncthreads();
    }
}

// The blocks a front's solves read, fetched into L2 ahead of use.
__device__ __forceinline__ void msolve_prefetch(const FrontDev& fd, int s) {
    const int f = fd.f[s], p = fd.p[s];
    prefetch_l2(fd.linv + fd.linv_off[s], sizeof(float) * p * p);
    prefetch_l2(fd.pool + fd.off[s], sizeof(float) * (size_t)p * f);
}

// Forward substitution L y = r for front s (one CTA), then z = D^-1 y.  y_s =
// L_ss^-1 w_s with the stored explicit inverse; the rows below accumulate
// -L_Us y_s into the front's update vector, which the parent adds in.  The
// children's update vectors are read through L2 (other CTAs of a tree-scheduled
// launch write them).
__device__ __forceinline__ void msolve_fwd_front(const FrontDev& fd, int s, float* __restrict__ w) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const float* F = fd.pool + fd.off[s];
    const float* X = fd.linv + fd.linv_off[s];
    const int f = fd.f[s], p = fd.p[s];
    const int base = 3 * fd.begin[s];
    float* y = w + f;
    float* red = y + f;                // [GV_MAXG][GV_ROWS] partial sums
    // w = the children's update entries (pull lists: children in order), then r
    // on the pivots -- the sums of a child-by-child scatter into zeroed storage
    const int* pp = fd.pull_ptr + fd.pull_off[s];
    for (int t = tid; t < f; t += nt) {
        const int node = t / 3, comp = t - 3 * node;
        float a = 0.0f;
        for (int e = pp[node]; e < pp[node + 1]; ++e) a += __ldcg(fd.acc + fd.pull_idx[e] + comp);
        if (t < p) a += fd.rvec[base + t];
        w[t] = a;
    }
    __syncthreads();
    cm_gemv(X, p, p, p, true, w, red, [&](int i, float t) { y[i] = t; });
    float* acc = fd.acc + fd.acc_off[s];
    cm_gemv(F + p, f, f - p, p, false, y, red, [&](int i, float t) { acc[i] = w[p + i] - t; });
    for (int t = tid; t < p; t += nt) fd.zvec[base + t] = y[t] / F[(long)t * f + t];
}

// Forward substitution over one level (CTA per front of sn_list).
__global__ void __launch_bounds__(FT) k_msolve_fwd(FrontDev fd, const int* __restrict__ sn_list,
                                                    const double* __restrict__ mask) {
    extern __shared__ float w[];
    const int s = sn_list[blockIdx.x];
    if (mask && mask[fd.sn_inst[s]] == 0.0) return;
    msolve_prefetch(fd, s);
    msolve_fwd_front(fd, s, w);
}

// Backward substitution L^T x = z for front s (one CTA), top-down: x_s =
// L_ss^-T (z_s - L_Us^T x_U).  One warp per row (lanes along the row), two rows
// per warp at a time; a row's sum does not depend on the CTA size.  x_U is read
// through L2 (the ancestors' CTAs of a tree-scheduled launch write it).
__device__ __forceinline__ void msolve_bwd_front(const FrontDev& fd, int s, float* __restrict__ sm) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const float* F = fd.pool + fd.off[s];
    const float* X = fd.linv + fd.linv_off[s];
    const int f = fd.f[s], p = fd.p[s], nu = f - p;
    const int base = 3 * fd.begin[s];
    float* w = sm;
    float* xu = sm + p;
    const int* un = fd.unode + fd.uptr[s];
    for (int t = tid; t < p; t += nt) w[t] = fd.zvec[base + t];
    for (int k = tid; k < nu; k += nt) xu[k] = __ldcg(fd.xvec + 3 * un[k / 3] + k % 3);
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    for (int t = warp; t < p; t += 2 * nw) {
        const int t2 = t + nw;
        const bool two = t2 < p;
        const float* r1 = F + (long)t * f + p;
        const float* r2 = F + (long)(two ? t2 : t) * f + p;
        float s1 = 0.0f, s2 = 0.0f;
        for (int k = lane; k < nu; k += 32) {
            const float x = xu[k];
            s1 += r1[k] * x;
            s2 += r2[k] * x;
        }
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            w[t] -= s1;
            if (two) w[t2] -= s2;
        }
    }
    __syncthreads();
    for (int i = warp; i < p; i += 2 * nw) {
        const int i2 = i + nw;
        const bool two = i2 < p;
        const float* c1 = X + (long)i * p;   // column i of L_ss^-1 = row i of L_ss^-T
        const float* c2 = X + (long)(two ? i2 : i) * p;
        float s1 = 0.0f, s2 = 0.0f;
        for (int k = i + lane; k < p; k += 32) s1 += c1[k] * w[k];
        if (two)
            for (int k = i2 + lane; k < p; k += 32) s2 += c2[k] * w[k];
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            fd.xvec[base + i] = s1;
            if (two) fd.xvec[base + i2] = s2;
        }
    }
}

// Backward substitution over one level (CTA per front of sn_list).
__global__ void __launch_bounds__(FT) k_msolve_bwd(FrontDev fd, const int* __restrict__ sn_list,
                                                    const double* __restrict__ mask) {
    extern __shared__ float sm[];
    const int s = sn_list[blockIdx.x];
    if (mask && mask[fd.sn_inst[s]] == 0.0) return;
    msolve_prefetch(fd, s);
    msolve_bwd_front(fd, s, sm);
}

// Tree-scheduled solves: one launch per sweep.  Persistent CTAs take the fronts
// of items[0 .. n_items) (a topological order, children first) from a ticket
// counter; the backward sweep takes them in reverse.  Before a front a CTA waits
// (bounded, dc_wait.cuh) for its children's done flags (forward) or its
// parent's (backward).  A front is only ever waited on by fronts of its own
// instance, and an instance is masked whole, so a masked front is skipped
// without a flag.  An item waits only on items with smaller tickets, held by
// CTAs already running, so the launch completes whatever the number resident.
// Threads per CTA of a tree-scheduled solve: the fronts on the dependency chain
// are the large ones, so wide CTAs pay (measured on the 256-cloth batch: 128
// threads 1.50 s, 256 threads 1.09 s, 512 threads 1.02 s of solves per bench step).
constexpr int MT = 512;

__device__ __forceinline__ int ms_take(const FrontDev& fd, int* ticket, int n_items, int* s_item) {
    if (threadIdx.x == 0) *s_item = dc_fault_set(fd.fault) ? n_items : atomicAdd(ticket, 1);
    __syncthreads();
    const int t = *s_item;
    __syncthreads();   // every thread has read the ticket before it is rewritten
    return t;
}

__global__ void __launch_bounds__(MT) k_msolve_fwd_tree(FrontDev fd, const int* __restrict__ items, int n_items,
                                                        const double* __restrict__ mask) {
    extern __shared__ float w[];
    __shared__ int s_item, s_ok;
    int* ticket = fd.sched;
    int* done = fd.sched + 1;
    for (;;) {
        const int t = ms_take(fd, ticket, n_items, &s_item);
        if (t >= n_items) return;
        const int s = items[t];
        if (mask && mask[fd.sn_inst[s]] == 0.0) continue;
        msolve_prefetch(fd, s);
        if (threadIdx.x == 0) {
            bool ok = true;
            for (int q = fd.cptr[s]; ok && q < fd.cptr[s + 1]; ++q) ok = dc_wait_flag(done + fd.child[q], fd.fault);
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) return;
        msolve_fwd_front(fd, s, w);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) dc_st_release(done + s, 1);
    }
}

__global__ void __launch_bounds__(MT) k_msolve_bwd_tree(FrontDev fd, const int* __restrict__ items, int n_items,
                                                        const double* __restrict__ mask) {
    extern __shared__ float sm[];
    __shared__ int s_item, s_ok;
    int* ticket = fd.sched + fd.S + 1;
    int* done = fd.sched + fd.S + 2;
    for (;;) {
        const int t = ms_take(fd, ticket, n_items, &s_item);
        if (t >= n_items) return;
        const int s = items[n_items - 1 - t];
        if (mask && mask[fd.sn_inst[s]] == 0.0) continue;
        msolve_prefetch(fd, s);
        if (threadIdx.x == 0) {
            const int par = fd.parent[s];
            s_ok = par < 0 || dc_wait_flag(done + par, fd.fault);
        }
        __syncthreads();
        if (!s_ok) return;
        msolve_bwd_front(fd, s, sm);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) dc_st_release(done + s, 1);
    }
}

// r = Pi_B w in single precision (DOF order 3*node + c).
__global__ void k_pre_in(int n, const int* __restrict__ type, const d4* __restrict__ nb, const d4* __restrict__ w,
                         float* __restrict__ r, const int* __restrict__ node_inst, const double* __restrict__ mask) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    if (mask && mask[node_inst[j]] == 0.0) return;
    d4 a = ld(w + j);
    double v[3] = {a.x, a.y, a.z};
    int ty = type[j];
    if (ty == 1) {
        v[0] = v[1] = v[2] = 0.0;
    } else if (ty == 2) {
        d4 q = ld(nb + j);
        double s = q.x * v[0] + q.y * v[1] + q.z * v[2];
        v[0] -= s * q.x; v[1] -= s * q.y; v[2] -= s * q.z;
    }
    r[3 * j] = (float)v[0];
    r[3 * j + 1] = (float)v[1];
    r[3 * j + 2] = (float)v[2];
}

// out = S_C x in double precision: stick -> 0, slip -> x - n ((n - mu t).x).
__global__ void k_pre_out(int n, const double* __restrict__ mu, const int* __restrict__ type, const d4* __restrict__ nb,
                          const d4* __restrict__ slip, const float* __restrict__ x, d4* __restrict__ out,
                          const int* __restrict__ node_inst, const double* __restrict__ mask) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    if (mask && mask[node_inst[j]] == 0.0) return;
    double v[3] = {(double)x[3 * j], (double)x[3 * j + 1], (double)x[3 * j + 2]};
    int ty = type[j];
    if (ty == 1) {
        v[0] = v[1] = v[2] = 0.0;
    } else if (ty == 2) {
        d4 q = ld(nb + j), sl = ld(slip + j);
        const double mj = mu[j];
        double cz = (q.x - mj * sl.x) * v[0] + (q.y - mj * sl.y) * v[1] + (q.z - mj * sl.z) * v[2];
        v[0] -= cz * q.x; v[1] -= cz * q.y; v[2] -= cz * q.z;
    }
    st(out + j, v[0], v[1], v[2]);
}

}  // namespace

// Shared memory of a factorisation CTA: the diagonal block, its inverse, the
// pivots and the transposed rows below the block (one panel width of the front),
// or the scratch of the explicit inverse of a pivot block of up to max_p rows.
// With tc, the tensor-core operand buffers come first.
size_t frontal_factor_smem(int max_f, int max_p, bool tc) {
    const size_t ldt = ((size_t)max_f + 7) / 8 * 8;
    size_t panel = (2 * (size_t)PB * LDS + PB + 3) / 4 * 4 + PB * ldt;
    size_t inverse = 2 * (size_t)PB * (max_p + 1) + (size_t)PB * PB;
    return ((tc ? TC_FLOATS : 0) + (panel > inverse ? panel : inverse)) * sizeof(float) + 64;
}

// Whether a level whose largest front has max_f unknowns uses the tensor-core
// trailing update (off for every level when DC_FRONT_FMA=1 is in the environment).
bool frontal_level_tc(int max_f) {
    static const bool off = [] {
        const char* e = getenv("DC_FRONT_FMA");
        return e && e[0] == '1';
    }();
    return !off && max_f >= TC_MIN_F;
}

// The same CTA with its panel and inverse scratch in global memory: the shared
// part, and the global floats per CTA (a multiple of 4).
size_t frontal_factor_smem_small(bool tc) {
    return ((tc ? TC_FLOATS : 0) + (2 * (size_t)PB * LDS + PB + 3) / 4 * 4) * sizeof(float) + 64;
}
long frontal_factor_gscr(int max_f, int max_p) {
    const long ldt = ((long)max_f + 7) / 8 * 8;
    const long panel = (long)PB * ldt, inverse = 2L * PB * (max_p + 1) + (long)PB * PB;
    return ((panel > inverse ? panel : inverse) + 3) / 4 * 4;
}

size_t frontal_solve_smem(int max_f) { return (2 * (size_t)max_f + GV_ROWS * GV_MAXG) * sizeof(float) + 64; }

// The dynamic shared-memory limit of the front kernels is a per-function
// attribute shared by every context of the process, so it only ever grows.
void frontal_plan(const HostFronts& fr, size_t smem_limit, long* gscr_floats, size_t* factor_bytes) {
    const int nl = (int)fr.lvl_ptr.size() - 1;
    *gscr_floats = 0;
    *factor_bytes = frontal_factor_smem_small(false);
    for (int l = 0; l < nl; ++l) {
        int mf = 0, mp = 0;
        for (int q = fr.lvl_ptr[l]; q < fr.lvl_ptr[l + 1]; ++q) {
            mf = std::max(mf, fr.f[fr.lvl_sn[q]]);
            mp = std::max(mp, fr.p[fr.lvl_sn[q]]);
        }
        const bool tc = frontal_level_tc(mf);
        const size_t need = frontal_factor_smem(mf, mp, tc);
        if (need <= smem_limit) {
            *factor_bytes = std::max(*factor_bytes, need);
        } else {
            *factor_bytes = std::max(*factor_bytes, frontal_factor_smem_small(tc));
            *gscr_floats = std::max(*gscr_floats, (long)(fr.lvl_ptr[l + 1] - fr.lvl_ptr[l]) * frontal_factor_gscr(mf, mp));
        }
    }
}

cudaError_t frontal_configure(size_t fb, int max_f) {
    static std::mutex mu;
    static size_t factor_bytes = 48 * 1024, solve_bytes = 48 * 1024;
    std::lock_guard<std::mutex> lock(mu);
    const size_t sb = frontal_solve_smem(max_f);
    if (fb > factor_bytes) {
        cudaError_t e = cudaFuncSetAttribute(k_front_level, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fb);
        if (e != cudaSuccess) return e;
        factor_bytes = fb;
    }
    if (sb > solve_bytes) {
        for (const void* k : {(const void*)k_msolve_fwd, (const void*)k_msolve_bwd, (const void*)k_msolve_fwd_tree,
                              (const void*)k_msolve_bwd_tree}) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
            if (e != cudaSuccess) return e;
        }
        solve_bytes = sb;
    }
    return cudaSuccess;
}

// One dense front through k_front_level: the test hook behind
// dc_debug_front_factor (synchronous; allocates and frees its own buffers).
dc_status frontal_debug_factor(int n, int p, const float* A, float* out, float* linv_out, int threads, int tc,
                               int use_gscr, std::string* err) {
    if (n < 1 || p < 1 || p > n || n > 4096 || (threads != 128 && threads != 256 && threads != 512)) {
        *err = "dc_debug_front_factor: needs 1 <= p <= n <= 4096 and 128, 256 or 512 threads";
        return DC_ERR_INVALID;
    }
    if (!A || !out) {
        *err = "dc_debug_front_factor: null A or out";
        return DC_ERR_INVALID;
    }
    const int nbk = (p + PB - 1) / PB;
    const long gsz = frontal_factor_gscr(n, p);
    const size_t smem = use_gscr ? frontal_factor_smem_small(tc != 0) : frontal_factor_smem(n, p, tc != 0);
    if (smem > 227 * 1024) {
        *err = "dc_debug_front_factor: front too large for shared memory; set use_gscr";
        return DC_ERR_INVALID;
    }
    // device image: ints [lvl_sn, f, p, cptr0, cptr1], long longs [off, binv_off, linv_off]
    int hi[5] = {0, n, p, 0, 0};
    long long hl[3] = {0, 0, 0};
    float tau = 1e-30f;
    int* di = nullptr;
    long long* dl = nullptr;
    float *pool = nullptr, *binv = nullptr, *linv = nullptr, *dtau = nullptr, *gscr = nullptr;
    unsigned long long* fault = nullptr;
    cudaError_t e = cudaSuccess;
    auto fail = [&](cudaError_t ce) {
        *err = std::string("dc_debug_front_factor: ") + cudaGetErrorString(ce);
        return DC_ERR_CUDA;
    };
    dc_status st = DC_OK;
    do {
        if ((e = cudaMalloc(&di, sizeof(hi))) || (e = cudaMalloc(&dl, sizeof(hl))) ||
            (e = cudaMalloc(&pool, sizeof(float) * (size_t)n * n)) ||
            (e = cudaMalloc(&binv, sizeof(float) * (size_t)nbk * PB * PB)) ||
            (e = cudaMalloc(&linv, sizeof(float) * (size_t)p * p)) || (e = cudaMalloc(&dtau, sizeof(float))) ||
            (e = cudaMalloc(&fault, sizeof(unsigned long long))) ||
            (use_gscr && (e = cudaMalloc(&gscr, sizeof(float) * (size_t)gsz)))) {
            st = fail(e);
            break;
        }
        if ((e = cudaMemcpy(di, hi, sizeof(hi), cudaMemcpyHostToDevice)) ||
            (e = cudaMemcpy(dl, hl, sizeof(hl), cudaMemcpyHostToDevice)) ||
            (e = cudaMemcpy(dtau, &tau, sizeof(float), cudaMemcpyHostToDevice)) ||
            (e = cudaMemcpy(pool, A, sizeof(float) * (size_t)n * n, cudaMemcpyHostToDevice)) ||
            (e = cudaMemset(fault, 0, sizeof(unsigned long long))) ||
            (e = frontal_configure(smem, n))) {
            st = fail(e);
            break;
        }
        FrontDev fd{};
        fd.S = 1;
        fd.max_f = n;
        fd.tau = dtau;
        fd.lvl_sn = di;
        fd.f = di + 1;
        fd.p = di + 2;
        fd.cptr = di + 3;
        fd.off = dl;
        fd.binv_off = dl + 1;
        fd.linv_off = dl + 2;
        fd.pool = pool;
        fd.binv = binv;
        fd.linv = linv;
        fd.fault = fault;
        dc_note_launch();
        k_front_level<<<1, threads, smem>>>(fd, 0, n, use_gscr ? gscr : nullptr, use_gscr ? gsz : 0L, tc ? 1 : 0);
        if ((e = cudaGetLastError()) || (e = cudaDeviceSynchronize())) {
            st = fail(e);
            break;
        }
        unsigned long long fl = 0;
        if ((e = cudaMemcpy(&fl, fault, sizeof(fl), cudaMemcpyDeviceToHost)) ||
            (e = cudaMemcpy(out, pool, sizeof(float) * (size_t)n * n, cudaMemcpyDeviceToHost)) ||
            (linv_out && (e = cudaMemcpy(linv_out, linv, sizeof(float) * (size_t)p * p, cudaMemcpyDeviceToHost)))) {
            st = fail(e);
            break;
        }
        if (fl) {
            *err = "dc_debug_front_factor: a tensor-core wait gave up";
            st = DC_ERR_TIMEOUT;
        }
    } while (false);
    cudaFree(di);
    cudaFree(dl);
    cudaFree(pool);
    cudaFree(binv);
    cudaFree(linv);
    cudaFree(dtau);
    cudaFree(fault);
    cudaFree(gscr);
    return st;
}

cudaError_t frontal_tree_grid(int max_f, int* grid_f, int* grid_b, size_t* smem_out) {
    const size_t smem = frontal_solve_smem(max_f);
    *smem_out = smem;
    int dev = 0, sms = 0, nf = 0, nb = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nf, k_msolve_fwd_tree, MT, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_msolve_bwd_tree, MT, smem);
    if (e != cudaSuccess) return e;
    *grid_f = sms * (nf > 0 ? nf : 1);
    *grid_b = sms * (nb > 0 ? nb : 1);
    return cudaSuccess;
}

// Threads per CTA for a level of cnt fronts whose largest has mf unknowns: small
// fronts get small CTAs (and, with the level's own shared-memory size, many CTAs
// per SM).  The kernel takes 128 registers a thread, so a 512-thread CTA fills an
// SM's register file; a level with at least four fronts per SM (two waves of two
// CTAs) uses 256 threads instead when two CTAs fit in shared memory, so that one
// CTA's serial phases (the diagonal block on one warp) overlap the other's
// updates.  With fewer fronts the halved CTAs only lengthen the one wave.  The
// results do not depend on the CTA size.
static int factor_threads(int mf, int mp, int cnt, int sms) {
    if (mf <= 96) return 128;
    if (mf <= 192) return 256;
    if (cnt >= 4 * sms && 2 * frontal_factor_smem(mf, mp, frontal_level_tc(mf)) <= 227 * 1024) return 256;
    // (levels on the global-scratch path keep FT2 threads)
    return FT2;
}
static int solve_threads(int mf) { return mf <= 64 ? 128 : (mf <= 128 ? 256 : (mf <= 256 ? 512 : FT)); }

void frontal_factorize(const DevMesh& dm, const AdjDev& ad, const FrontDev& fd, const int* lvl_ptr, int nlev,
                       const int* lvl_maxf, const int* lvl_maxp, cudaStream_t s, KTimer* kt) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (kt) kt->begin(DC_KT_ASSEMBLE);
    cudaMemsetAsync(fd.pool, 0, sizeof(float) * fd.pool_size, s);
    dc_note_launch();
    k_pairs<<<nblk(fd.NP, 128), 128, 0, s>>>(dm, ad, fd);
    if (kt) kt->end(DC_KT_ASSEMBLE);
    for (int l = 0; l < nlev; ++l) {
        int cnt = lvl_ptr[l + 1] - lvl_ptr[l];
        if (cnt > 0) {
            const int mf = lvl_maxf[l];
            dc_note_launch();
            if (kt) kt->begin(DC_KT_FRONT);
            const int mp = lvl_maxp[l];
            const bool tc = frontal_level_tc(mf);
            if (frontal_factor_smem(mf, mp, tc) <= fd.smem_limit) {
                k_front_level<<<cnt, factor_threads(mf, mp, cnt, sms), frontal_factor_smem(mf, mp, tc), s>>>(
                    fd, lvl_ptr[l], mf, nullptr, 0L, tc ? 1 : 0);
            } else {   // fronts too large for shared memory: panel scratch in fd.gscr
                k_front_level<<<cnt, FT2, frontal_factor_smem_small(tc), s>>>(fd, lvl_ptr[l], mf, fd.gscr,
                                                                            frontal_factor_gscr(mf, mp), tc ? 1 : 0);
            }
            if (kt) kt->end(DC_KT_FRONT);
        }
    }
}

void frontal_precond(const AdjDev& ad, const FrontDev& fd, const int* lvl_ptr, int nlev, const int* lvl_maxf,
                     int n_free, const d4* w, d4* out, cudaStream_t s, KTimer* kt, const int* act_sn,
                     const int* act_ptr, const int* act_tq, int n_act_tq) {
    dc_note_launch();
    k_pre_in<<<nblk(n_free, 128), 128, 0, s>>>(n_free, ad.type, ad.nb, w, fd.rvec, ad.node_inst, ad.mask);
    if (fd.tree) {
        const int* items = act_tq ? act_tq : fd.tq;
        const int n = act_tq ? n_act_tq : fd.S;
        if (n > 0) {
            cudaMemsetAsync(fd.sched, 0, sizeof(int) * 2 * ((size_t)fd.S + 1), s);
            if (kt) kt->begin(DC_KT_MSOLVE);
            dc_note_launch();
            k_msolve_fwd_tree<<<n < fd.tree_grid_f ? n : fd.tree_grid_f, MT, fd.tree_smem, s>>>(fd, items, n, ad.mask);
            dc_note_launch();
            k_msolve_bwd_tree<<<n < fd.tree_grid_b ? n : fd.tree_grid_b, MT, fd.tree_smem, s>>>(fd, items, n, ad.mask);
            if (kt) kt->end(DC_KT_MSOLVE);
        }
        dc_note_launch();
        k_pre_out<<<nblk(n_free, 128), 128, 0, s>>>(n_free, ad.mu, ad.type, ad.nb, ad.slip, fd.xvec, out,
                                                      ad.node_inst, ad.mask);
        return;
    }
    // level l's fronts: the compacted list of the active instances' fronts, or all of them
    auto level = [&](int l, int& cnt) -> const int* {
        if (act_sn) {
            cnt = act_ptr[l + 1] - act_ptr[l];
            return act_sn + act_ptr[l];
        }
        cnt = lvl_ptr[l + 1] - lvl_ptr[l];
        return fd.lvl_sn + lvl_ptr[l];
    };
    for (int l = 0; l < nlev; ++l) {
        int cnt;
        const int* sn = level(l, cnt);
        if (cnt > 0) {
            const int mf = lvl_maxf[l];
            dc_note_launch();
            if (kt) kt->begin(DC_KT_MSOLVE);
            k_msolve_fwd<<<cnt, solve_threads(mf), frontal_solve_smem(mf), s>>>(fd, sn, ad.mask);
            if (kt) kt->end(DC_KT_MSOLVE);
        }
    }
    for (int l = nlev - 1; l >= 0; --l) {
        int cnt;
        const int* sn = level(l, cnt);
        if (cnt > 0) {
            const int mf = lvl_maxf[l];
            dc_note_launch();
            if (kt) kt->begin(DC_KT_MSOLVE);
            k_msolve_bwd<<<cnt, solve_threads(mf), frontal_solve_smem(mf), s>>>(fd, sn, ad.mask);
            if (kt) kt->end(DC_KT_MSOLVE);
        }
    }
    dc_note_launch();
    k_pre_out<<<nblk(n_free, 128), 128, 0, s>>>(n_free, ad.mu, ad.type, ad.nb, ad.slip, fd.xvec, out,
                                                  ad.node_inst, ad.mask);
}
