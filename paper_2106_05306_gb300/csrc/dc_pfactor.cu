// Numeric Cholesky of the PD matrix P on the GPU (dc_params.factor_on_gpu):
// Eq. pd_global's "prefactorised" P = M + h^2 sum_i w_i A_i^T A_i, as a
// multifrontal FP64 factorisation over the supernodes of the nested-dissection
// ordering, written straight into the supernodal panels of the substitution
// (global_solver 1).  The host keeps the ordering and the symbolic structure
// (they depend on the mesh only); the values, which change with every new
// stiffness, density or h, are computed here.
//
// Fronts are node-level (P = P_s kron I3, so the scalar factor is enough) and
// column-major in a temporary pool: front s has fs = ns + nu rows (its own ns
// nodes, then its update nodes U_s) and ld = fs.  Per tree level, leaves first,
// one CTA per front: the children's update blocks are added in through the
// child-to-parent position maps, the first ns columns are factorised (right-
// looking, one column at a time), and the panel (ns + nu) x ns, the inverse of
// its top block, and the transposed copies the backward sweep reads are written.
// The trailing block is the front's update block for its parent.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "dc_ctx.h"

namespace {

inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

__device__ __forceinline__ void g_row(const d4& g, int a, double& g0, double& g1) {
    if (a == 1) { g0 = g.x; g1 = g.y; }
    else if (a == 2) { g0 = g.z; g1 = g.w; }
    else { g0 = -(g.x + g.z); g1 = -(g.y + g.w); }
}

// P's lower entries into the fronts: the mass on the diagonal plus h^2 times the
// stretch (w_t g_a . g_b) and bending (w_b l_bi l_bj) contributions of the pair.
__global__ void k_pf_assemble(DevMesh dm, FrontDev fd, const long long* __restrict__ dst, double h2,
                              double* __restrict__ pool) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= fd.NP) return;
    const int i = fd.pr_i[id], j = fd.pr_j[id];
    double acc = 0.0;
    for (int k = fd.pr_cptr[id]; k < fd.pr_cptr[id + 1]; ++k) {
        const int code = fd.pr_code[k];
        if (code >= 0) {
            const int t = code / 9, a = (code / 3) % 3, b = code % 3;
            const d4 g = dm.G[t];
            double ga0, ga1, gb0, gb1;
            g_row(g, a, ga0, ga1);
            g_row(g, b, gb0, gb1);
            acc += dm.wt[t] * (ga0 * gb0 + ga1 * gb1);
        } else {
            acc += dm.wb[-code - 1] * fd.pr_coef[k];
        }
    }
    pool[dst[id]] = (i == j ? dm.mass[i] : 0.0) + h2 * acc;
}

struct PanelOut {
    double* panel;
    double* xinv;
    double* pant;
    double* xinvt;
    const long long* poff;
    const long long* xoff;
    const long long* toff;
};

__global__ void __launch_bounds__(256) k_pf_front(FrontDev fd, const long long* __restrict__ offN, int lvl_begin,
                                                  double* __restrict__ pool, PanelOut out,
                                                  unsigned long long* __restrict__ not_spd) {
    __shared__ double dk;
    const int s = fd.lvl_sn[lvl_begin + blockIdx.x];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int ns = fd.p[s] / 3, fs = fd.f[s] / 3, nu = fs - ns;
    double* F = pool + offN[s];
    // extend-add of the children's update blocks (lower triangles; the position
    // maps are increasing, so lower entries land on lower entries)
    for (int q = fd.cptr[s]; q < fd.cptr[s + 1]; ++q) {
        const int c = fd.child[q];
        const double* Fc = pool + offN[c];
        const int nsc = fd.p[c] / 3, fsc = fd.f[c] / 3, nuc = fsc - nsc;
        const int* map = fd.cmap + fd.uptr[c];
        for (int b = warp; b < nuc; b += nw) {
            const double* src = Fc + (long)(nsc + b) * fsc + nsc;
            double* dst = F + (long)map[b] * fs;
            for (int a = b + lane; a < nuc; a += 32) dst[map[a]] += src[a];
        }
        __syncthreads();
    }
    // partial Cholesky of the first ns columns
    for (int k = 0; k < ns; ++k) {
        if (tid == 0) {
            double d = F[(long)k * fs + k];
            if (!(d > 0.0)) {
                atomicExch(not_spd, 1ull);
                d = 1.0;
            }
            dk = sqrt(d);
            F[(long)k * fs + k] = dk;
        }
        __syncthreads();
        const double l = dk;
        double* colk = F + (long)k * fs;
        for (int i = k + 1 + tid; i < fs; i += nt) colk[i] = colk[i] / l;
        __syncthreads();
        for (int j = k + 1 + warp; j < fs; j += nw) {
            const double ljk = colk[j];
            double* colj = F + (long)j * fs;
            for (int i = j + lane; i < fs; i += 32) colj[i] -= colk[i] * ljk;
        }
        __syncthreads();
    }
    // panel (zero above the diagonal) and the transposed update rows
    double* pan = out.panel + out.poff[s];
    for (long e = tid; e < (long)ns * fs; e += nt) {
        const int c = (int)(e / fs), r = (int)(e % fs);
        pan[e] = r >= c ? F[e] : 0.0;
    }
    double* T = out.pant + out.toff[s];
    for (long e = tid; e < (long)ns * nu; e += nt) {
        const int c = (int)(e % ns), k = (int)(e / ns);
        T[e] = F[(long)c * fs + ns + k];
    }
    // X = inverse of the lower-triangular top block, column c by one thread:
    // X[r][c] = (delta_rc - sum_{k=c}^{r-1} L[r][k] X[k][c]) / L[r][r]
    double* X = out.xinv + out.xoff[s];
    for (int c = tid; c < ns; c += nt) {
        double* xc = X + (long)c * ns;
        for (int r = 0; r < c; ++r) xc[r] = 0.0;
        for (int r = c; r < ns; ++r) {
            double t = (r == c) ? 1.0 : 0.0;
            for (int k = c; k < r; ++k) t -= F[(long)k * fs + r] * xc[k];
            xc[r] = t / F[(long)r * fs + r];
        }
    }
    __syncthreads();
    double* XT = out.xinvt + out.xoff[s];
    for (long e = tid; e < (long)ns * ns; e += nt) {
        const int c = (int)(e / ns), r = (int)(e % ns);
        XT[(long)r * ns + c] = X[e];
    }
}

}  // namespace

// Factorises P on the context's stream into the panels of c->dm.ps (synchronous).
dc_status gpu_factor_P(dc_ctx* c, const HostFronts& frm, double h) {
    const int S = frm.S;
    // node-level front offsets and the destination of every matrix pair
    std::vector<long long> offN(S + 1, 0);
    for (int s = 0; s < S; ++s) {
        const long long fs = frm.f[s] / 3;
        offN[s + 1] = offN[s] + fs * fs;
    }
    std::vector<int> sn_of(c->hm.m_free, -1);
    for (int s = 0; s < S; ++s)
        for (int j = frm.begin[s]; j < frm.end[s]; ++j) sn_of[j] = s;
    const size_t NP = frm.pr_i.size();
    std::vector<long long> dst(NP);
    for (size_t id = 0; id < NP; ++id) {
        const int s = sn_of[frm.pr_j[id]];
        const long long rel = frm.pr_dst[id] - frm.off[s], f = frm.f[s];
        const long long pj = rel / (3 * f), pi = (rel % f) / 3;
        dst[id] = offN[s] + pj * (f / 3) + pi;
    }
    Pool tmp;
    double* pool = nullptr;
    long long *d_off = nullptr, *d_dst = nullptr;
    dc_status st;
    if ((st = dalloc(c, tmp, &pool, (size_t)std::max<long long>(offN[S], 1))) ||
        (st = upload(c, tmp, &d_off, offN)) || (st = upload(c, tmp, &d_dst, dst))) {
        free_pool(c, tmp);
        return st;
    }
    cudaStream_t s = c->stream;
    CK(cudaMemsetAsync(c->counters + 5, 0, sizeof(unsigned long long), s));
    dc_note_launch();
    k_pf_assemble<<<nblk((long)NP, 256), 256, 0, s>>>(c->dm, c->fdv, d_dst, h * h, pool);
    PanelOut out{const_cast<double*>(c->dm.ps.panel), const_cast<double*>(c->dm.ps.xinv),
                 const_cast<double*>(c->dm.ps.pant), const_cast<double*>(c->dm.ps.xinvt), c->dm.ps.poff,
                 c->dm.ps.xoff, c->dm.ps.toff};
    const int nl = (int)frm.lvl_ptr.size() - 1;
    for (int l = 0; l < nl; ++l) {
        const int cnt = frm.lvl_ptr[l + 1] - frm.lvl_ptr[l];
        if (cnt <= 0) continue;
        dc_note_launch();
        k_pf_front<<<cnt, 256, 0, s>>>(c->fdv, d_off, frm.lvl_ptr[l], pool, out, c->counters + 5);
    }
    unsigned long long flag = 0;
    CK(cudaMemcpyAsync(&flag, c->counters + 5, sizeof(flag), cudaMemcpyDeviceToHost, s));
    CK(ctx_sync(c, s));
    CK(cudaGetLastError());
    free_pool(c, tmp);
    if (flag) {
        c->err = "dc_set_params: P is not positive definite (a pivot <= 0 in the GPU factorisation)";
        return DC_ERR_NOT_SPD;
    }
    return DC_OK;
}
