// C ABI of libdc: context management, the forward step / rollout, and the
// checkpointed backward pass with the flexible-GMRES adjoint solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "dc_adjoint.h"
#include "dc_internal.h"

namespace {

std::string g_create_err;

struct StepRec {
    int* contact = nullptr;
    int* case_ = nullptr;
    d4* nb = nullptr;
    d4* f = nullptr;
};

}  // namespace

void KTimer::begin(int c) {
    if (c != cls || cls == 0) return;
    if (ev.empty()) {
        ev.resize(2 * 4096);
        for (auto& e : ev) cudaEventCreate(&e);
    }
    if (used + 2 > (int)ev.size()) flush();
    cudaEventRecord(ev[used], stream);
}

void KTimer::end(int c) {
    if (c != cls || cls == 0) return;
    cudaEventRecord(ev[used + 1], stream);
    used += 2;
    ++launches;
}

void KTimer::flush() {
    if (used == 0) return;
    cudaEventSynchronize(ev[used - 1]);
    for (int i = 0; i < used; i += 2) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, ev[i], ev[i + 1]) == cudaSuccess) ms += t;
    }
    used = 0;
}

void KTimer::release() {
    for (auto& e : ev) cudaEventDestroy(e);
    ev.clear();
    used = 0;
}

struct dc_ctx {
    cudaStream_t stream = nullptr;
    std::string err;
    KTimer kt;
    double front_flops = 0.0;
    HostMesh hm;
    HostFactor hf;
    bool have_params = false;
    dc_params prm{};
    DevParams dp{};
    DevMesh dm{};
    std::vector<void*> mesh_allocs, factor_allocs, work_allocs, ck_allocs, seg_allocs, adj_allocs, front_allocs;
    HostFronts fr;
    FrontDev fdv{};
    int nlev = 0;
    int* d_int2ext = nullptr;
    // forward work
    d4 *xa = nullptr, *va = nullptr, *xb = nullptr, *vb = nullptr, *v = nullptr, *b = nullptr, *y = nullptr;
    d4 *c1 = nullptr, *c2 = nullptr, *bu = nullptr, *ind = nullptr;
    double* cc = nullptr;
    StepRec scratch;
    double* stage = nullptr;   // [m][3] staging for host/device conversion
    double* stage2 = nullptr;
    unsigned long long* counters = nullptr;
    // rollout checkpoints
    int ck_n_steps = -1, ck_every = 1, ck_cap = 0;
    d4* ck = nullptr;          // [(cap)][2][m]
    // backward segment buffers
    int seg_cap = 0;
    d4* segX = nullptr;        // [(cap+1)][m]
    d4* segV = nullptr;
    std::vector<StepRec> seg_rec;
    // adjoint buffers
    int adj_restart_cap = 0;
    AdjDev ad{};                  // the slot in use by the GMRES of the current adjoint step
    AdjDev ads[2]{};              // per-step adjoint data, two slots (even / odd steps)
    FrontDev fds[2]{};            // numeric fronts, two slots
    cudaStream_t stream2 = nullptr;   // assembles and factorises the next step's fronts
    cudaEvent_t ev_fact[2]{}, ev_free[2]{}, ev_seg = nullptr;
    KTimer kt2;
    d4 *gx = nullptr, *gv = nullptr, *gx2 = nullptr, *gv2 = nullptr, *g = nullptr, *rhs = nullptr, *z = nullptr;
    d4 *x1 = nullptr, *r1 = nullptr, *x2 = nullptr, *r2 = nullptr, *ytmp = nullptr, *wv = nullptr, *E = nullptr;
    d4 *resid = nullptr;
    double *V = nullptr, *Zb = nullptr, *dcoef = nullptr, *dcoef2 = nullptr, *dnorm = nullptr, *partial = nullptr;
    double *dparam_acc = nullptr, *dparam_part = nullptr;
    double* hpin = nullptr;    // pinned host scratch
    // stats
    long long steps = 0, adj_steps = 0, adj_iters = 0, adj_max_seen = 0, adj_noncv = 0;
    double adj_last_res = 0.0;
    long long n_factorisations = 0;
};

namespace {

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            c->err = std::string("CUDA error: ") + cudaGetErrorString(e_) + " at " #call;     \
            return (e_ == cudaErrorMemoryAllocation) ? DC_ERR_OOM : DC_ERR_CUDA;              \
        }                                                                                     \
    } while (0)

template <class T>
dc_status dalloc(dc_ctx* c, std::vector<void*>& pool, T** p, size_t count, bool zero = true) {
    void* q = nullptr;
    size_t bytes = std::max<size_t>(count * sizeof(T), 32);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        c->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return DC_ERR_OOM;
    }
    if (zero) cudaMemset(q, 0, bytes);
    pool.push_back(q);
    *p = reinterpret_cast<T*>(q);
    return DC_OK;
}

void free_pool(std::vector<void*>& pool) {
    for (void* p : pool) cudaFree(p);
    pool.clear();
}

template <class T>
dc_status upload(dc_ctx* c, std::vector<void*>& pool, T** p, const std::vector<T>& h) {
    dc_status s = dalloc(c, pool, p, h.size(), false);
    if (s) return s;
    if (!h.empty()) CK(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return DC_OK;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

#define RET(x)                      \
    do {                            \
        dc_status s_ = (x);         \
        if (s_ != DC_OK) return s_; \
    } while (0)

// Copy an [m][3] argument into an internal d4 vector.
dc_status load_vec(dc_ctx* c, const double* ext, d4* out, bool& host_io) {
    const int m = c->hm.m;
    const double* src = ext;
    if (!is_device_ptr(ext)) {
        host_io = true;
        CK(cudaMemcpyAsync(c->stage, ext, sizeof(double) * 3 * m, cudaMemcpyDefault, c->stream));
        src = c->stage;
    }
    launch_permute_in(src, out, c->d_int2ext, m, c->stream);
    return DC_OK;
}

dc_status store_vec(dc_ctx* c, const d4* in, double* ext, bool& host_io) {
    const int m = c->hm.m;
    if (is_device_ptr(ext)) {
        launch_permute_out(in, ext, c->d_int2ext, m, c->stream);
    } else {
        host_io = true;
        launch_permute_out(in, c->stage2, c->d_int2ext, m, c->stream);
        CK(cudaMemcpyAsync(ext, c->stage2, sizeof(double) * 3 * m, cudaMemcpyDefault, c->stream));
    }
    return DC_OK;
}

dc_status alloc_rec(dc_ctx* c, std::vector<void*>& pool, StepRec& r) {
    const int mf = c->hm.m_free;
    RET(dalloc(c, pool, &r.contact, mf));
    RET(dalloc(c, pool, &r.case_, mf));
    RET(dalloc(c, pool, &r.nb, mf));
    RET(dalloc(c, pool, &r.f, mf));
    return DC_OK;
}

// One time step (Sec. 3.2) on internal vectors; writes the contact record into r.
void run_step(dc_ctx* c, const d4* xin, const d4* vin, d4* xout, d4* vout, StepRec& r, bool count = true) {
    cudaStream_t s = c->stream;
    const DevMesh& dm = c->dm;
    const DevParams& P = c->dp;
    launch_detect(dm, P, xin, vin, r.contact, r.nb, r.f, c->ind, s);
    cudaMemsetAsync(r.case_, 0, sizeof(int) * dm.m_free, s);
    // compliance c_j = h (P^-1 1_I)_j of the step's contact set (reading R5)
    launch_solve_fwd(dm, c->ind, c->y, s);
    launch_solve_bwd(dm, P, c->y, nullptr, 2, nullptr, nullptr, nullptr, nullptr, nullptr, c->cc, s);
    cudaMemcpyAsync(c->v, vin, sizeof(d4) * dm.m, cudaMemcpyDeviceToDevice, s);
    KTimer& kt = c->kt;
    for (int k = 0; k < c->prm.n_pd_iters; ++k) {
        kt.begin(DC_KT_LOCAL);
        launch_local(dm, P, xin, c->v, c->c1, c->c2, c->bu, s);
        kt.end(DC_KT_LOCAL);
        kt.begin(DC_KT_GATHER);
        launch_gather_rhs(dm, P, vin, c->c1, c->c2, c->bu, r.f, c->b, s);
        kt.end(DC_KT_GATHER);
        kt.begin(DC_KT_SOLVE_FWD);
        launch_solve_fwd(dm, c->b, c->y, s);
        kt.end(DC_KT_SOLVE_FWD);
        kt.begin(DC_KT_SOLVE_BWD);
        launch_solve_bwd(dm, P, c->y, c->v, 1, r.contact, r.nb, c->cc, r.f, r.case_, nullptr, s);
        kt.end(DC_KT_SOLVE_BWD);
    }
    launch_finalize(dm, P, xin, c->v, xout, s);
    if (vout != c->v) cudaMemcpyAsync(vout, c->v, sizeof(d4) * dm.m, cudaMemcpyDeviceToDevice, s);
    if (count) {
        launch_count_cases(r.contact, r.case_, dm.m_free, c->counters, s);
        c->steps++;
    }
}

dc_status ensure_checkpoints(dc_ctx* c, int n_ck) {
    if (n_ck <= c->ck_cap) return DC_OK;
    free_pool(c->ck_allocs);
    RET(dalloc(c, c->ck_allocs, &c->ck, (size_t)n_ck * 2 * c->hm.m));
    c->ck_cap = n_ck;
    return DC_OK;
}

dc_status ensure_segment(dc_ctx* c, int k) {
    if (k <= c->seg_cap) return DC_OK;
    free_pool(c->seg_allocs);
    c->seg_rec.assign(k, StepRec{});
    RET(dalloc(c, c->seg_allocs, &c->segX, (size_t)(k + 1) * c->hm.m));
    RET(dalloc(c, c->seg_allocs, &c->segV, (size_t)(k + 1) * c->hm.m));
    for (int i = 0; i < k; ++i) RET(alloc_rec(c, c->seg_allocs, c->seg_rec[i]));
    c->seg_cap = k;
    return DC_OK;
}

dc_status ensure_adjoint(dc_ctx* c) {
    int mr = std::max(1, std::min(256, c->prm.adj_restart));
    if (c->V && mr <= c->adj_restart_cap) return DC_OK;
    free_pool(c->adj_allocs);
    const int m = c->hm.m, mf = c->hm.m_free, T = c->hm.T;
    auto& P = c->adj_allocs;
    d4 *c1, *c2, *bu;
    RET(dalloc(c, P, &c1, T));
    RET(dalloc(c, P, &c2, T));
    RET(dalloc(c, P, &bu, m));
    for (int k = 0; k < 2; ++k) {
        AdjDev& a = c->ads[k];
        RET(dalloc(c, P, &a.tr0, T));
        RET(dalloc(c, P, &a.tr1, T));
        RET(dalloc(c, P, &a.tr2, T));
        RET(dalloc(c, P, &a.bq, m));
        RET(dalloc(c, P, &a.dinv, 3 * (size_t)mf));
        RET(dalloc(c, P, &a.slip, mf));
        RET(dalloc(c, P, &a.type, mf));
        a.c1 = c1;
        a.c2 = c2;
        a.bu = bu;
    }
    c->ad = c->ads[0];
    if (!c->stream2) {
        CK(cudaStreamCreateWithFlags(&c->stream2, cudaStreamNonBlocking));
        for (int k = 0; k < 2; ++k) {
            CK(cudaEventCreateWithFlags(&c->ev_fact[k], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&c->ev_free[k], cudaEventDisableTiming));
        }
        CK(cudaEventCreateWithFlags(&c->ev_seg, cudaEventDisableTiming));
        c->kt2.stream = c->stream2;
        c->kt2.cls = c->kt.cls;
    }
    d4** vecs[] = {&c->gx, &c->gv, &c->gx2, &c->gv2, &c->g, &c->rhs, &c->z, &c->x1,
                   &c->r1, &c->x2, &c->r2, &c->ytmp, &c->wv, &c->E, &c->resid};
    for (d4** p : vecs) RET(dalloc(c, P, p, m));
    RET(dalloc(c, P, &c->V, (size_t)(mr + 1) * 4 * m));
    RET(dalloc(c, P, &c->Zb, (size_t)mr * 4 * m));
    RET(dalloc(c, P, &c->dcoef, mr + 2));
    RET(dalloc(c, P, &c->dcoef2, mr + 2));
    RET(dalloc(c, P, &c->dnorm, 4));
    RET(dalloc(c, P, &c->partial, (size_t)(mr + 2) * adj_red_blocks()));
    RET(dalloc(c, P, &c->dparam_acc, 4));
    RET(dalloc(c, P, &c->dparam_part, 3 * (size_t)adj_red_blocks()));
    c->adj_restart_cap = mr;
    return DC_OK;
}

inline d4* vcol(double* base, int j, int m) { return reinterpret_cast<d4*>(base + (size_t)j * 4 * m); }

// Preconditioner K(w) -> out: block inverse, projected P^-1, block inverse.
void precond(dc_ctx* c, const d4* w, d4* out) {
    cudaStream_t s = c->stream;
    const DevMesh& dm = c->dm;
    const AdjDev& ad = c->ad;
    if (c->prm.adj_precond == 0) {
        frontal_precond(ad, c->fdv, c->fr.lvl_ptr.data(), c->nlev, c->fr.max_f, dm.m_free, w, out, s, &c->kt);
        return;
    }
    adj_dplus(dm, ad, nullptr, w, c->x1, s);
    adj_apply_H(dm, ad, 1, c->x1, w, c->r1, s);
    adj_solve_project(dm, ad, c->r1, c->ytmp, c->x1, c->x2, s);
    adj_apply_H(dm, ad, 1, c->x2, w, c->r2, s);
    adj_dplus(dm, ad, c->x2, c->r2, out, s);
}

dc_status dot_host(dc_ctx* c, const double* a, const double* b, long n, double* out) {
    adj_mdot(a, 0, 1, b, n, c->partial, c->dnorm, c->stream);
    CK(cudaMemcpyAsync(c->hpin, c->dnorm, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *out = c->hpin[0];
    return DC_OK;
}

// Flexible GMRES for Pi_B H z = rhs with z in null(C^T).  Returns the
// iteration count in *iters and the final relative residual in *rel.
dc_status gmres(dc_ctx* c, int* iters, double* rel) {
    cudaStream_t s = c->stream;
    const int m = c->hm.m, mf = c->hm.m_free;
    const long n = 4L * mf;
    const int mr = std::max(1, std::min(256, c->prm.adj_restart));
    const int maxit = std::max(1, c->prm.adj_max_iters);
    const double tol = c->prm.adj_tol;
    double* zz = reinterpret_cast<double*>(c->z);
    double* rr = reinterpret_cast<double*>(c->r1);
    CK(cudaMemsetAsync(c->z, 0, sizeof(d4) * m, s));
    double beta0;
    RET(dot_host(c, reinterpret_cast<double*>(c->rhs), reinterpret_cast<double*>(c->rhs), n, &beta0));
    beta0 = std::sqrt(beta0);
    *iters = 0;
    *rel = 0.0;
    if (!(beta0 > 0.0)) return DC_OK;
    if (!std::isfinite(beta0)) {
        c->err = "non-finite adjoint right-hand side";
        return DC_ERR_NONFINITE;
    }
    std::vector<double> H((size_t)(mr + 1) * mr), cs(mr), sn(mr), gg(mr + 1), yv(mr);
    int total = 0;
    // residual r = rhs (z = 0)
    CK(cudaMemcpyAsync(c->r1, c->rhs, sizeof(d4) * m, cudaMemcpyDeviceToDevice, s));
    double res = beta0, prev_cycle = 0.0;
    const bool debug = std::getenv("DC_DEBUG_GMRES") != nullptr;
    for (int cycle = 0;; ++cycle) {
        double beta;
        RET(dot_host(c, rr, rr, n, &beta));
        beta = std::sqrt(beta);
        res = beta;
        if (debug) std::fprintf(stderr, "[dc gmres] cycle %d iters %d true rel residual %.3e\n", cycle, total, beta / beta0);
        if (beta <= tol * beta0 || total >= maxit) break;
        // a restart that did not halve the true residual means the rounding floor
        // (about eps * cond(H)) has been reached: stop there
        if (cycle > 0 && beta > 0.5 * prev_cycle) break;
        prev_cycle = beta;
        adj_scale(rr, 1.0 / beta, c->V, n, s);
        std::fill(gg.begin(), gg.end(), 0.0);
        gg[0] = beta;
        int used = 0;
        bool done = false;
        for (int j = 0; j < mr; ++j) {
            d4* vj = vcol(c->V, j, m);
            d4* zj = vcol(c->Zb, j, m);
            precond(c, vj, zj);
            adj_apply_H(c->dm, c->ad, 0, zj, nullptr, c->wv, s);
            double* w = reinterpret_cast<double*>(c->wv);
            adj_mdot(c->V, 4L * m, j + 1, w, n, c->partial, c->dcoef, s);
            adj_vupdate(c->V, 4L * m, j + 1, c->dcoef, w, n, -1.0, s);
            adj_mdot(c->V, 4L * m, j + 1, w, n, c->partial, c->dcoef2, s);
            adj_vupdate(c->V, 4L * m, j + 1, c->dcoef2, w, n, -1.0, s);
            adj_mdot(w, 0, 1, w, n, c->partial, c->dnorm, s);
            CK(cudaMemcpyAsync(c->hpin, c->dcoef, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(c->hpin + 260, c->dcoef2, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(c->hpin + 520, c->dnorm, sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            double* hc = &H[(size_t)j * (mr + 1)];
            for (int i = 0; i <= j; ++i) hc[i] = c->hpin[i] + c->hpin[260 + i];
            double hn = std::sqrt(std::max(c->hpin[520], 0.0));
            hc[j + 1] = hn;
            if (!std::isfinite(hn)) {
                c->err = "non-finite value in the adjoint iteration";
                return DC_ERR_NONFINITE;
            }
            if (hn > 0.0) adj_scale(w, 1.0 / hn, reinterpret_cast<double*>(vcol(c->V, j + 1, m)), n, s);
            for (int i = 0; i < j; ++i) {
                double t = cs[i] * hc[i] + sn[i] * hc[i + 1];
                hc[i + 1] = -sn[i] * hc[i] + cs[i] * hc[i + 1];
                hc[i] = t;
            }
            double den = std::hypot(hc[j], hc[j + 1]);
            cs[j] = den > 0 ? hc[j] / den : 1.0;
            sn[j] = den > 0 ? hc[j + 1] / den : 0.0;
            hc[j] = den;
            hc[j + 1] = 0.0;
            gg[j + 1] = -sn[j] * gg[j];
            gg[j] = cs[j] * gg[j];
            ++total;
            used = j + 1;
            res = std::fabs(gg[j + 1]);
            if (res <= tol * beta0 || total >= maxit || hn == 0.0) {
                done = true;
                break;
            }
        }
        for (int i = used - 1; i >= 0; --i) {
            double t = gg[i];
            for (int k = i + 1; k < used; ++k) t -= H[(size_t)k * (mr + 1) + i] * yv[k];
            yv[i] = t / H[(size_t)i * (mr + 1) + i];
        }
        for (int i = 0; i < used; ++i) c->hpin[i] = yv[i];
        CK(cudaMemcpyAsync(c->dcoef, c->hpin, sizeof(double) * used, cudaMemcpyHostToDevice, s));
        adj_vupdate(c->Zb, 4L * m, used, c->dcoef, zz, n, 1.0, s);
        // true residual r = rhs - Pi_B H z
        adj_apply_H(c->dm, c->ad, 1, c->z, c->rhs, c->r1, s);
        if (done && total >= maxit) {
            RET(dot_host(c, rr, rr, n, &res));
            res = std::sqrt(res);
            break;
        }
    }
    *iters = total;
    *rel = res / beta0;
    return DC_OK;
}

// Per-step adjoint data of step q into slot k: the element linearisation, node
// types and (with the multifrontal preconditioner) the factorised fronts.  Runs on
// stream2 so that it overlaps the GMRES of the step after q.
void prepare_step(dc_ctx* c, int q, int k, cudaStream_t s) {
    AdjDev& ad = c->ads[k];
    const StepRec& r = c->seg_rec[q];
    const int m = c->hm.m;
    ad.h = c->prm.h;
    ad.mu = c->prm.mu;
    ad.contact = r.contact;
    ad.case_ = r.case_;
    ad.nb = r.nb;
    ad.f = r.f;
    adj_setup(c->dm, ad, c->segX + (size_t)(q + 1) * m, c->segV + (size_t)(q + 1) * m, s);
    if (c->prm.adj_precond == 0) {
        frontal_factorize(c->dm, ad, c->fds[k], c->fr.lvl_ptr.data(), c->nlev, c->fr.max_f, s,
                          s == c->stream ? &c->kt : &c->kt2);
        c->n_factorisations++;
    }
}

// One adjoint step from slot k: (gx, gv) at n+1 -> (gx2, gv2) at n, parameter
// terms into dparam_acc.
dc_status adjoint_step(dc_ctx* c, const d4* x_n, const d4* x1, const d4* v1, int k, bool& noncv) {
    cudaStream_t s = c->stream;
    c->ad = c->ads[k];
    c->fdv = c->fds[k];
    AdjDev& ad = c->ad;
    adj_rhs(c->dm, ad, c->gx, c->gv, c->g, c->rhs, s);
    int it = 0;
    double rel = 0.0;
    RET(gmres(c, &it, &rel));
    c->adj_steps++;
    c->adj_iters += it;
    c->adj_max_seen = std::max<long long>(c->adj_max_seen, it);
    c->adj_last_res = rel;
    if (!(rel <= c->prm.adj_tol * 1.0000001)) {
        c->adj_noncv++;
        noncv = true;
    }
    adj_apply_H(c->dm, ad, 3, c->z, nullptr, c->E, s);
    adj_apply_H(c->dm, ad, 2, c->z, c->g, c->resid, s);
    adj_outputs(c->dm, ad, c->dp, c->z, c->E, c->resid, x_n, v1, c->gx, c->gx2, c->gv2, s);
    adj_params(c->dm, ad, c->z, x1, c->dparam_part, c->dparam_acc, s);
    CK(cudaEventRecord(c->ev_free[k], s));
    std::swap(c->gx, c->gx2);
    std::swap(c->gv, c->gv2);
    return DC_OK;
}

bool finite_params(const dc_params& p) {
    const double v[] = {p.k_stretch, p.k_bend, p.density, p.mu, p.h, p.gravity[0], p.gravity[1], p.gravity[2],
                        p.contact_margin, p.adj_tol};
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

}  // namespace

extern "C" {

void dc_default_params(dc_params* p) {
    std::memset(p, 0, sizeof(*p));
    p->k_stretch = 1e3;
    p->k_bend = 1e-3;
    p->density = 0.1;
    p->mu = 0.3;
    p->h = 1.0 / 120.0;
    p->gravity[1] = -9.8;
    p->contact_margin = 1e-6;
    p->adj_tol = 1e-10;
    p->n_pd_iters = 20;
    p->adj_max_iters = 2000;
    p->adj_restart = 200;
    p->checkpoint_every = 1;
    p->n_obstacles = 0;
}

dc_status dc_create_mesh(dc_ctx** out, int32_t n_nodes, const double* rest_pos, int32_t n_tris,
                         const int32_t* tris, int32_t n_pins, const int32_t* pins, void* stream) {
    if (!out || !rest_pos || !tris || n_pins < 0 || (n_pins > 0 && !pins)) {
        g_create_err = "dc_create_mesh: null argument";
        return DC_ERR_INVALID;
    }
    *out = nullptr;
    dc_ctx* c = new dc_ctx();
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    c->kt.stream = c->stream;
    std::string e = dc_build_mesh(c->hm, n_nodes, rest_pos, n_tris, tris, n_pins, pins);
    if (!e.empty()) {
        g_create_err = "dc_create_mesh: " + e;
        delete c;
        return DC_ERR_INVALID;
    }
    const HostMesh& hm = c->hm;
    const int m = hm.m, T = hm.T;
    auto& P = c->mesh_allocs;
    auto fail = [&](dc_status s) {
        g_create_err = c->err;
        free_pool(c->mesh_allocs);
        delete c;
        return s;
    };
    dc_status s;
    std::vector<int4> tri4(T);
    std::vector<d4> G4(T);
    std::vector<double> area = hm.area;
    for (int t = 0; t < T; ++t) {
        tri4[t] = make_int4(hm.tri[3 * t], hm.tri[3 * t + 1], hm.tri[3 * t + 2], 0);
        G4[t] = d4{hm.G[4 * t], hm.G[4 * t + 1], hm.G[4 * t + 2], hm.G[4 * t + 3]};
    }
    std::vector<d4> qr(m);
    for (int i = 0; i < m; ++i) qr[i] = d4{hm.qrest[3 * i], hm.qrest[3 * i + 1], hm.qrest[3 * i + 2], 0.0};
    // node -> triangle incidences and transpose bending stencils
    std::vector<int> iptr(m + 1, 0), iidx, tbptr(m + 1, 0), tbidx;
    std::vector<double> tbval;
    {
        std::vector<std::vector<int>> inc(m);
        for (int t = 0; t < T; ++t)
            for (int a = 0; a < 3; ++a) inc[hm.tri[3 * t + a]].push_back(3 * t + a);
        for (int i = 0; i < m; ++i) {
            iptr[i + 1] = iptr[i] + (int)inc[i].size();
            iidx.insert(iidx.end(), inc[i].begin(), inc[i].end());
        }
        std::vector<std::vector<std::pair<int, double>>> tb(m);
        for (int b = 0; b < m; ++b)
            for (int k = hm.bptr[b]; k < hm.bptr[b + 1]; ++k) tb[hm.bidx[k]].push_back({b, hm.bval[k]});
        for (int i = 0; i < m; ++i) {
            tbptr[i + 1] = tbptr[i] + (int)tb[i].size();
            for (auto& e2 : tb[i]) {
                tbidx.push_back(e2.first);
                tbval.push_back(e2.second);
            }
        }
    }
    int4* d_tri;
    d4 *d_G, *d_qr;
    double *d_area, *d_bval, *d_abar, *d_sb, *d_tbval;
    int *d_bptr, *d_bidx, *d_iptr, *d_iidx, *d_tbptr, *d_tbidx;
    if ((s = upload(c, P, &d_tri, tri4)) || (s = upload(c, P, &d_G, G4)) || (s = upload(c, P, &d_area, area)) ||
        (s = upload(c, P, &d_bptr, hm.bptr)) || (s = upload(c, P, &d_bidx, hm.bidx)) ||
        (s = upload(c, P, &d_bval, hm.bval)) || (s = upload(c, P, &d_abar, hm.abar)) ||
        (s = upload(c, P, &d_sb, hm.sb)) || (s = upload(c, P, &d_qr, qr)) || (s = upload(c, P, &d_iptr, iptr)) ||
        (s = upload(c, P, &d_iidx, iidx)) || (s = upload(c, P, &d_tbptr, tbptr)) ||
        (s = upload(c, P, &d_tbidx, tbidx)) || (s = upload(c, P, &d_tbval, tbval)) ||
        (s = upload(c, P, &c->d_int2ext, hm.int2ext)))
        return fail(s);
    DevMesh& dm = c->dm;
    dm.m = m;
    dm.m_free = hm.m_free;
    dm.T = T;
    dm.tri = d_tri;
    dm.G = d_G;
    dm.area = d_area;
    dm.bptr = d_bptr;
    dm.bidx = d_bidx;
    dm.bval = d_bval;
    dm.abar = d_abar;
    dm.sb = d_sb;
    dm.qrest = d_qr;
    dm.iptr = d_iptr;
    dm.iidx = d_iidx;
    dm.tbptr = d_tbptr;
    dm.tbidx = d_tbidx;
    dm.tbval = d_tbval;
    // work buffers
    auto& W = c->work_allocs;
    d4** vecs[] = {&c->xa, &c->va, &c->xb, &c->vb, &c->v, &c->b, &c->y, &c->bu, &c->ind};
    for (d4** p : vecs)
        if ((s = dalloc(c, W, p, m))) return fail(s);
    if ((s = dalloc(c, W, &c->c1, T)) || (s = dalloc(c, W, &c->c2, T)) || (s = dalloc(c, W, &c->cc, m)) ||
        (s = dalloc(c, W, &c->stage, 3 * (size_t)m)) || (s = dalloc(c, W, &c->stage2, 3 * (size_t)m)) ||
        (s = dalloc(c, W, &c->counters, 4)) || (s = alloc_rec(c, W, c->scratch)))
        return fail(s);
    if (cudaMallocHost(&c->hpin, 1024 * sizeof(double)) != cudaSuccess) {
        c->err = "cudaMallocHost failed";
        return fail(DC_ERR_OOM);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        c->err = "device error during dc_create_mesh";
        return fail(DC_ERR_CUDA);
    }
    *out = c;
    return DC_OK;
}

dc_status dc_set_params(dc_ctx* c, const dc_params* p) {
    if (!c || !p) return DC_ERR_INVALID;
    if (!finite_params(*p) || !(p->h > 0) || p->k_stretch < 0 || p->k_bend < 0 || !(p->density > 0) ||
        p->mu < 0 || p->n_pd_iters < 0 || p->n_obstacles < 0 || p->n_obstacles > DC_MAX_OBSTACLES ||
        p->checkpoint_every < 1 || p->adj_max_iters < 1 || p->adj_restart < 1 || !(p->adj_tol > 0) ||
        p->adj_precond < 0 || p->adj_precond > 1) {
        c->err = "dc_set_params: invalid or non-finite parameter";
        return DC_ERR_INVALID;
    }
    dc_params q = *p;
    DevParams dp{};
    for (int o = 0; o < q.n_obstacles; ++o) {
        dc_obstacle& ob = q.obstacles[o];
        for (int k = 0; k < 7; ++k)
            if (!std::isfinite(ob.p[k])) {
                c->err = "dc_set_params: non-finite obstacle";
                return DC_ERR_INVALID;
            }
        if (ob.kind == DC_PLANE) {
            double nn = std::sqrt(ob.p[0] * ob.p[0] + ob.p[1] * ob.p[1] + ob.p[2] * ob.p[2]);
            if (!(nn > 0)) {
                c->err = "dc_set_params: zero plane normal";
                return DC_ERR_INVALID;
            }
            for (int k = 0; k < 3; ++k) ob.p[k] /= nn;
            ob.p[3] /= nn;
        } else if (ob.kind == DC_SPHERE) {
            if (!(ob.p[3] > 0)) {
                c->err = "dc_set_params: sphere radius must be positive";
                return DC_ERR_INVALID;
            }
        } else if (ob.kind == DC_CAPSULE) {
            double L = std::fabs(ob.p[3] - ob.p[0]) + std::fabs(ob.p[4] - ob.p[1]) + std::fabs(ob.p[5] - ob.p[2]);
            if (!(ob.p[6] > 0) || !(L > 0)) {
                c->err = "dc_set_params: bad capsule";
                return DC_ERR_INVALID;
            }
        } else {
            c->err = "dc_set_params: unknown obstacle kind";
            return DC_ERR_INVALID;
        }
        dp.kind[o] = ob.kind;
        for (int k = 0; k < 7; ++k) dp.op[o][k] = ob.p[k];
    }
    dp.n_obst = q.n_obstacles;
    dp.k_stretch = q.k_stretch;
    dp.k_bend = q.k_bend;
    dp.mu = q.mu;
    dp.h = q.h;
    for (int k = 0; k < 3; ++k) dp.g[k] = q.gravity[k];
    dp.delta = q.contact_margin;

    const HostMesh& hm = c->hm;
    std::vector<double> mass(hm.m), wt(hm.T), wb(hm.m);
    for (int i = 0; i < hm.m; ++i) {
        mass[i] = q.density * hm.abar[i];
        wb[i] = q.k_bend * hm.abar[i];
    }
    for (int t = 0; t < hm.T; ++t) wt[t] = q.k_stretch * hm.area[t];
    CK(cudaStreamSynchronize(c->stream));
    HostFactor hf;
    std::string err;
    dc_status s = dc_build_factor(hm, q, mass, hf, err);
    if (s) {
        c->err = "dc_set_params: " + err;
        return s;
    }
    free_pool(c->factor_allocs);
    auto& P = c->factor_allocs;
    double *d_mass, *d_wt, *d_wb, *d_fval, *d_kval;
    int *d_fptr, *d_fidx, *d_kptr, *d_kidx, *d_long, *d_short;
    std::vector<int> long_rows, short_rows;
    for (int i = 0; i < hm.m_free; ++i)
        (hf.fptr[i + 1] - hf.fptr[i] > 1024 ? long_rows : short_rows).push_back(i);
    if ((s = upload(c, P, &d_mass, mass)) || (s = upload(c, P, &d_wt, wt)) || (s = upload(c, P, &d_wb, wb)) ||
        (s = upload(c, P, &d_fptr, hf.fptr)) || (s = upload(c, P, &d_fidx, hf.fidx)) ||
        (s = upload(c, P, &d_fval, hf.fval)) || (s = upload(c, P, &d_kptr, hf.bptr)) ||
        (s = upload(c, P, &d_kidx, hf.bidx)) || (s = upload(c, P, &d_kval, hf.bval)) ||
        (s = upload(c, P, &d_long, long_rows)) || (s = upload(c, P, &d_short, short_rows)))
        return s;
    c->dm.n_long = (int)long_rows.size();
    c->dm.n_short = (int)short_rows.size();
    c->dm.long_rows = d_long;
    c->dm.short_rows = d_short;
    c->dm.mass = d_mass;
    c->dm.wt = d_wt;
    c->dm.wb = d_wb;
    c->dm.fptr = d_fptr;
    c->dm.fidx = d_fidx;
    c->dm.fval = d_fval;
    c->dm.kptr = d_kptr;
    c->dm.kidx = d_kidx;
    c->dm.kval = d_kval;
    // multifrontal structure for the adjoint preconditioner
    HostFronts fr;
    std::string fe = dc_build_fronts(hm, hf, fr);
    if (!fe.empty()) {
        c->err = "dc_set_params: " + fe;
        return DC_ERR_INVALID;
    }
    int dev = 0, smem_optin = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (frontal_factor_smem(fr.max_f) > (size_t)smem_optin) {
        c->err = "dc_set_params: the largest front (" + std::to_string(fr.max_f) +
                 " unknowns) exceeds the shared memory of one CTA";
        return DC_ERR_INVALID;
    }
    CK(frontal_configure(fr.max_f));
    free_pool(c->front_allocs);
    {
        auto& F = c->front_allocs;
        FrontDev fd{};
        fd.S = fr.S;
        fd.NP = (int)fr.pr_i.size();
        fd.tau = (float)(1e-7 * hf.max_diag);
        fd.max_f = fr.max_f;
        fd.pool_size = fr.pool_size;
        int *d_begin, *d_f, *d_p, *d_uptr, *d_unode, *d_cptr, *d_child, *d_cmap, *d_lvl, *d_pi, *d_pj, *d_pld, *d_pcp,
            *d_pcode;
        long long *d_off, *d_acc_off, *d_pdst, *d_binv_off, *d_linv_off;
        double* d_pcoef;
        if ((s = upload(c, F, &d_begin, fr.begin)) || (s = upload(c, F, &d_f, fr.f)) || (s = upload(c, F, &d_p, fr.p)) ||
            (s = upload(c, F, &d_off, fr.off)) || (s = upload(c, F, &d_acc_off, fr.acc_off)) ||
            (s = upload(c, F, &d_binv_off, fr.binv_off)) || (s = dalloc(c, F, &fd.binv, (size_t)fr.binv_size)) ||
            (s = upload(c, F, &d_linv_off, fr.linv_off)) || (s = dalloc(c, F, &fd.linv, (size_t)fr.linv_size)) ||
            (s = upload(c, F, &d_uptr, fr.uptr)) || (s = upload(c, F, &d_unode, fr.unode)) ||
            (s = upload(c, F, &d_cptr, fr.cptr)) || (s = upload(c, F, &d_child, fr.child)) ||
            (s = upload(c, F, &d_cmap, fr.cmap)) || (s = upload(c, F, &d_lvl, fr.lvl_sn)) ||
            (s = upload(c, F, &d_pi, fr.pr_i)) || (s = upload(c, F, &d_pj, fr.pr_j)) ||
            (s = upload(c, F, &d_pdst, fr.pr_dst)) || (s = upload(c, F, &d_pld, fr.pr_ld)) ||
            (s = upload(c, F, &d_pcp, fr.pr_cptr)) || (s = upload(c, F, &d_pcode, fr.pr_code)) ||
            (s = upload(c, F, &d_pcoef, fr.pr_coef)) || (s = dalloc(c, F, &fd.pool, (size_t)fr.pool_size)) ||
            (s = dalloc(c, F, &fd.acc, (size_t)fr.acc_size)) || (s = dalloc(c, F, &fd.rvec, 3 * (size_t)hm.m_free)) ||
            (s = dalloc(c, F, &fd.zvec, 3 * (size_t)hm.m_free)) || (s = dalloc(c, F, &fd.xvec, 3 * (size_t)hm.m_free)))
            return s;
        fd.begin = d_begin;
        fd.f = d_f;
        fd.p = d_p;
        fd.off = d_off;
        fd.acc_off = d_acc_off;
        fd.binv_off = d_binv_off;
        fd.linv_off = d_linv_off;
        fd.uptr = d_uptr;
        fd.unode = d_unode;
        fd.cptr = d_cptr;
        fd.child = d_child;
        fd.cmap = d_cmap;
        fd.lvl_sn = d_lvl;
        fd.pr_i = d_pi;
        fd.pr_j = d_pj;
        fd.pr_dst = d_pdst;
        fd.pr_ld = d_pld;
        fd.pr_cptr = d_pcp;
        fd.pr_code = d_pcode;
        fd.pr_coef = d_pcoef;
        c->fdv = fd;
        c->fds[0] = fd;
        c->fds[1] = fd;   // second slot: its own numeric storage, shared structure
        if ((s = dalloc(c, F, &c->fds[1].pool, (size_t)fr.pool_size)) ||
            (s = dalloc(c, F, &c->fds[1].binv, (size_t)fr.binv_size)) ||
            (s = dalloc(c, F, &c->fds[1].linv, (size_t)fr.linv_size)))
            return s;
    }
    c->nlev = (int)fr.lvl_ptr.size() - 1;
    c->front_flops = 0.0;
    for (int q = 0; q < fr.S; ++q)
        for (int k = 0; k < fr.p[q]; ++k) {
            double r = fr.f[q] - k - 1;
            c->front_flops += r + r * (r + 1.0);
        }
    c->fr = std::move(fr);
    c->hf = std::move(hf);
    c->prm = q;
    c->dp = dp;
    c->have_params = true;
    c->ck_n_steps = -1;
    return DC_OK;
}

dc_status dc_step(dc_ctx* c, const double* x_n, const double* v_n, double* x_np1, double* v_np1) {
    if (!c) return DC_ERR_INVALID;
    if (!c->have_params) {
        c->err = "dc_step: call dc_set_params first";
        return DC_ERR_STATE;
    }
    if (!x_n || !v_n || !x_np1 || !v_np1) {
        c->err = "dc_step: null array";
        return DC_ERR_INVALID;
    }
    bool host_io = false;
    RET(load_vec(c, x_n, c->xa, host_io));
    RET(load_vec(c, v_n, c->va, host_io));
    launch_zero_pins(c->va, c->hm.m_free, c->hm.m, c->stream);
    run_step(c, c->xa, c->va, c->xb, c->vb, c->scratch);
    RET(store_vec(c, c->xb, x_np1, host_io));
    RET(store_vec(c, c->vb, v_np1, host_io));
    CK(cudaGetLastError());
    if (host_io) CK(cudaStreamSynchronize(c->stream));
    return DC_OK;
}

dc_status dc_rollout(dc_ctx* c, int32_t n_steps, const double* x0, const double* v0, double* x_final,
                     double* v_final, double* traj_x) {
    if (!c) return DC_ERR_INVALID;
    if (!c->have_params) {
        c->err = "dc_rollout: call dc_set_params first";
        return DC_ERR_STATE;
    }
    if (n_steps < 0 || !x0 || !v0 || !x_final || !v_final) {
        c->err = "dc_rollout: bad arguments";
        return DC_ERR_INVALID;
    }
    const int m = c->hm.m;
    const int k = c->prm.checkpoint_every;
    const int n_ck = n_steps / k + 1;
    RET(ensure_checkpoints(c, n_ck));
    bool host_io = false;
    d4* X = c->ck;              // checkpoint 0 holds (x0, v0)
    d4* Vv = c->ck + m;
    RET(load_vec(c, x0, X, host_io));
    RET(load_vec(c, v0, Vv, host_io));
    launch_zero_pins(Vv, c->hm.m_free, m, c->stream);
    bool traj_dev = traj_x && is_device_ptr(traj_x);
    if (traj_x) {
        bool h2 = false;
        RET(store_vec(c, X, traj_x, h2));
        host_io |= h2;
    }
    d4 *cx = X, *cv = Vv;
    d4* bufx[2] = {c->xa, c->xb};
    d4* bufv[2] = {c->va, c->vb};
    for (int s = 0; s < n_steps; ++s) {
        d4 *nx, *nv;
        if ((s + 1) % k == 0) {
            nx = c->ck + (size_t)((s + 1) / k) * 2 * m;
            nv = nx + m;
        } else {
            nx = bufx[s & 1];
            nv = bufv[s & 1];
            if (nx == cx) {
                nx = bufx[(s + 1) & 1];
                nv = bufv[(s + 1) & 1];
            }
        }
        run_step(c, cx, cv, nx, nv, c->scratch);
        if (traj_x) {
            bool h2 = false;
            RET(store_vec(c, nx, traj_x + (size_t)(s + 1) * 3 * m, h2));
            host_io |= h2;
        }
        cx = nx;
        cv = nv;
    }
    (void)traj_dev;
    RET(store_vec(c, cx, x_final, host_io));
    RET(store_vec(c, cv, v_final, host_io));
    CK(cudaGetLastError());
    c->ck_n_steps = n_steps;
    c->ck_every = k;
    if (host_io) CK(cudaStreamSynchronize(c->stream));
    return DC_OK;
}

dc_status dc_backward(dc_ctx* c, const double* dL_dx_final, const double* dL_dv_final, const double* dL_dtraj_x,
                      double* dL_dx0, double* dL_dv0, double* dL_dparams) {
    if (!c) return DC_ERR_INVALID;
    if (c->ck_n_steps < 0) {
        c->err = "dc_backward: no rollout to differentiate (call dc_rollout after dc_set_params)";
        return DC_ERR_STATE;
    }
    if (!dL_dx_final || !dL_dx0 || !dL_dv0 || !dL_dparams) {
        c->err = "dc_backward: null array";
        return DC_ERR_INVALID;
    }
    const int N = c->ck_n_steps, k = c->ck_every, m = c->hm.m;
    cudaStream_t s = c->stream;
    RET(ensure_segment(c, k));
    RET(ensure_adjoint(c));
    bool host_io = false;
    RET(load_vec(c, dL_dx_final, c->gx, host_io));
    if (dL_dv_final)
        RET(load_vec(c, dL_dv_final, c->gv, host_io));
    else
        CK(cudaMemsetAsync(c->gv, 0, sizeof(d4) * m, s));
    launch_zero_pins(c->gv, c->hm.m_free, m, s);
    const double* traj = dL_dtraj_x;
    double* traj_dev = nullptr;
    std::vector<void*> tmp;
    if (traj && !is_device_ptr(traj)) {
        RET(dalloc(c, tmp, &traj_dev, (size_t)(N + 1) * 3 * m, false));
        CK(cudaMemcpyAsync(traj_dev, traj, sizeof(double) * (N + 1) * 3 * m, cudaMemcpyHostToDevice, s));
        traj = traj_dev;
        host_io = true;
    }
    CK(cudaMemsetAsync(c->dparam_acc, 0, 4 * sizeof(double), s));
    bool noncv = false;
    dc_status st = DC_OK;
    int n_seg = (N + k - 1) / k;
    for (int seg = n_seg - 1; seg >= 0 && st == DC_OK; --seg) {
        int s0 = seg * k, s1 = std::min(N, s0 + k);
        const d4* ckx = c->ck + (size_t)seg * 2 * m;
        CK(cudaMemcpyAsync(c->segX, ckx, sizeof(d4) * m, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(c->segV, ckx + m, sizeof(d4) * m, cudaMemcpyDeviceToDevice, s));
        for (int q = 0; q < s1 - s0; ++q)
            run_step(c, c->segX + (size_t)q * m, c->segV + (size_t)q * m, c->segX + (size_t)(q + 1) * m,
                     c->segV + (size_t)(q + 1) * m, c->seg_rec[q], false);
        // step q's data is prepared on stream2 while the GMRES of step q+1 runs on
        // the main stream; slot (s0 + q) % 2 alternates between consecutive steps
        CK(cudaEventRecord(c->ev_seg, s));
        CK(cudaStreamWaitEvent(c->stream2, c->ev_seg, 0));
        {
            const int q = s1 - s0 - 1, k2 = (s0 + q) % 2;
            CK(cudaStreamWaitEvent(c->stream2, c->ev_free[k2], 0));
            prepare_step(c, q, k2, c->stream2);
            CK(cudaEventRecord(c->ev_fact[k2], c->stream2));
        }
        for (int q = s1 - s0 - 1; q >= 0; --q) {
            const int k2 = (s0 + q) % 2;
            if (q > 0) {
                const int kn = (s0 + q - 1) % 2;
                CK(cudaStreamWaitEvent(c->stream2, c->ev_free[kn], 0));
                prepare_step(c, q - 1, kn, c->stream2);
                CK(cudaEventRecord(c->ev_fact[kn], c->stream2));
            }
            CK(cudaStreamWaitEvent(s, c->ev_fact[k2], 0));
            if (traj) adj_add_ext(c->gx, traj + (size_t)(s0 + q + 1) * 3 * m, c->d_int2ext, m, s);
            st = adjoint_step(c, c->segX + (size_t)q * m, c->segX + (size_t)(q + 1) * m,
                              c->segV + (size_t)(q + 1) * m, k2, noncv);
            if (st) break;
        }
    }
    if (st == DC_OK) {
        if (traj) adj_add_ext(c->gx, traj, c->d_int2ext, m, s);
        RET(store_vec(c, c->gx, dL_dx0, host_io));
        RET(store_vec(c, c->gv, dL_dv0, host_io));
        if (is_device_ptr(dL_dparams)) {
            CK(cudaMemcpyAsync(dL_dparams, c->dparam_acc, 3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
        } else {
            CK(cudaMemcpyAsync(dL_dparams, c->dparam_acc, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
            host_io = true;
        }
    }
    CK(cudaStreamSynchronize(s));
    if (c->stream2) CK(cudaStreamSynchronize(c->stream2));
    free_pool(tmp);
    CK(cudaGetLastError());
    if (st) return st;
    if (noncv) {
        c->err = "dc_backward: an adjoint step reached adj_max_iters above adj_tol";
        return DC_ERR_NONCONVERGED;
    }
    return DC_OK;
}

dc_status dc_global_solve(dc_ctx* c, const double* rhs, double* out) {
    if (!c) return DC_ERR_INVALID;
    if (!c->have_params) {
        c->err = "dc_global_solve: call dc_set_params first";
        return DC_ERR_STATE;
    }
    if (!rhs || !out) {
        c->err = "dc_global_solve: null array";
        return DC_ERR_INVALID;
    }
    bool host_io = false;
    RET(load_vec(c, rhs, c->b, host_io));
    launch_solve_fwd(c->dm, c->b, c->y, c->stream);
    CK(cudaMemsetAsync(c->v, 0, sizeof(d4) * c->hm.m, c->stream));
    launch_solve_bwd(c->dm, c->dp, c->y, c->v, 0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, c->stream);
    RET(store_vec(c, c->v, out, host_io));
    CK(cudaGetLastError());
    if (host_io) CK(cudaStreamSynchronize(c->stream));
    return DC_OK;
}

dc_status dc_get_stats(dc_ctx* c, dc_stats* o) {
    if (!c || !o) return DC_ERR_INVALID;
    CK(cudaStreamSynchronize(c->stream));
    unsigned long long cnt[4] = {0, 0, 0, 0};
    CK(cudaMemcpy(cnt, c->counters, sizeof(cnt), cudaMemcpyDeviceToHost));
    std::memset(o, 0, sizeof(*o));
    o->steps = c->steps;
    o->contacts_takeoff = (int64_t)cnt[0];
    o->contacts_stick = (int64_t)cnt[1];
    o->contacts_slip = (int64_t)cnt[2];
    o->adj_steps = c->adj_steps;
    o->adj_iters = c->adj_iters;
    o->adj_max_iters_seen = c->adj_max_seen;
    o->adj_nonconverged = c->adj_noncv;
    o->adj_last_residual = c->adj_last_res;
    o->factor_nnz = c->hf.colptr.empty() ? 0 : c->hf.colptr.back();
    o->solve_nnz = (int64_t)c->hf.fval.size() + (int64_t)c->hf.bval.size();
    o->n_free = c->hm.m_free;
    o->nd_levels = c->hm.nd_depth + 1;
    c->kt.flush();
    c->kt2.flush();
    o->kernel_launches = dc_launch_count();
    o->timer_ms = c->kt.ms + c->kt2.ms;
    o->timer_launches = c->kt.launches + c->kt2.launches;
    o->fwd_solve_nnz = (int64_t)c->hf.fval.size();
    o->bwd_solve_nnz = (int64_t)c->hf.bval.size();
    o->front_flops = c->front_flops;
    o->front_levels = c->nlev;
    o->n_supernodes = c->fr.S;
    o->factorisations = c->n_factorisations;
    return DC_OK;
}

dc_status dc_set_kernel_timer(dc_ctx* c, int32_t kernel_class) {
    if (!c) return DC_ERR_INVALID;
    if (kernel_class < DC_KT_NONE || kernel_class > DC_KT_MSOLVE) {
        c->err = "dc_set_kernel_timer: unknown kernel class";
        return DC_ERR_INVALID;
    }
    c->kt.flush();
    c->kt2.flush();
    c->kt.cls = c->kt2.cls = kernel_class;
    c->kt.ms = c->kt2.ms = 0.0;
    c->kt.launches = c->kt2.launches = 0;
    return DC_OK;
}

dc_status dc_sync(dc_ctx* c) {
    if (!c) return DC_ERR_INVALID;
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaGetLastError());
    return DC_OK;
}

void dc_destroy(dc_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    if (c->stream2) cudaStreamSynchronize(c->stream2);
    c->kt.release();
    c->kt2.release();
    for (int k = 0; k < 2; ++k) {
        if (c->ev_fact[k]) cudaEventDestroy(c->ev_fact[k]);
        if (c->ev_free[k]) cudaEventDestroy(c->ev_free[k]);
    }
    if (c->ev_seg) cudaEventDestroy(c->ev_seg);
    if (c->stream2) cudaStreamDestroy(c->stream2);
    free_pool(c->adj_allocs);
    free_pool(c->seg_allocs);
    free_pool(c->ck_allocs);
    free_pool(c->work_allocs);
    free_pool(c->factor_allocs);
    free_pool(c->front_allocs);
    free_pool(c->mesh_allocs);
    if (c->hpin) cudaFreeHost(c->hpin);
    delete c;
}

const char* dc_last_error(dc_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

}  // extern "C"

// Read-only accessors used by dc_static_solve.cu.
bool dc_ctx_ready(const dc_ctx* c) { return c->have_params; }
const DevMesh& dc_ctx_mesh(const dc_ctx* c) { return c->dm; }
const DevParams& dc_ctx_params(const dc_ctx* c) { return c->dp; }
const int* dc_ctx_int2ext(const dc_ctx* c) { return c->d_int2ext; }
cudaStream_t dc_ctx_stream(const dc_ctx* c) { return c->stream; }
void dc_ctx_set_error(dc_ctx* c, const std::string& msg) { c->err = msg; }

extern "C" {

}  // extern "C"
