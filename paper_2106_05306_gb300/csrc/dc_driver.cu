// Host driver of a context: the forward time step and rollout (optionally as
// replayed CUDA graphs), checkpoint recomputation, the per-step adjoint with
// its batched flexible GMRES, and the block-size autotuner.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "dc_ctx.h"

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

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

dc_status alloc_rec(dc_ctx* c, Pool& pool, StepRec& r) {
    const int mf = c->hm.m_free;
    RET(dalloc(c, pool, &r.contact, mf));
    RET(dalloc(c, pool, &r.case_, mf));
    RET(dalloc(c, pool, &r.nb, mf));
    RET(dalloc(c, pool, &r.f, mf));
    return DC_OK;
}

// Copy an [m][3] argument into an internal d4 vector.
dc_status load_vec(dc_ctx* c, const double* ext, d4* out, bool& host_io) {
    const int m = c->hm.m;
    const double* src = ext;
    if (!is_device_ptr(ext)) {
        host_io = true;
        CK(cudaMemcpyAsync(c->stage, ext, sizeof(double) * 3 * m, cudaMemcpyDefault, c->stream));
        src = c->stage;
    }
    launch_permute_in(src, out, c->d_int2ext, m, c->layout, c->stream);
    return DC_OK;
}

dc_status store_vec(dc_ctx* c, const d4* in, double* ext, bool& host_io) {
    const int m = c->hm.m;
    if (is_device_ptr(ext)) {
        launch_permute_out(in, ext, c->d_int2ext, m, c->layout, c->stream);
    } else {
        host_io = true;
        launch_permute_out(in, c->stage2, c->d_int2ext, m, c->layout, c->stream);
        CK(cudaMemcpyAsync(ext, c->stage2, sizeof(double) * 3 * m, cudaMemcpyDefault, c->stream));
    }
    return DC_OK;
}

void run_step(dc_ctx* c, const d4* xin, const d4* vin, d4* xout, d4* vout, StepRec& r, bool count, int step,
              const int* step_base) {
    cudaStream_t s = c->stream;
    const DevMesh& dm = c->dm;
    const DevParams& P = c->dp;
    launch_detect(dm, P, xin, vin, r.contact, r.nb, r.f, c->ind, s);
    cudaMemsetAsync(r.case_, 0, sizeof(int) * dm.m_free, s);
    // compliance of the per-node contact solve (reading R5): c_j = h (P^-1 1_I)_j
    // of the step's contact set, or a constant per node for the other choices
    const double* cc = P.ccon;
    if (P.compliance == DC_COMPLIANCE_ROWSUM) {
        if (!launch_solve_sweeps(dm, P, c->ind, c->y, nullptr, 2, nullptr, nullptr, nullptr, nullptr, nullptr, c->cc,
                                 s)) {
            launch_solve_fwd(dm, c->ind, c->y, s);
            launch_solve_bwd(dm, P, c->y, nullptr, 2, nullptr, nullptr, nullptr, nullptr, nullptr, c->cc, s);
        }
        cc = c->cc;
    }
    cudaMemcpyAsync(c->v, vin, sizeof(d4) * dm.m, cudaMemcpyDeviceToDevice, s);
    KTimer& kt = c->kt;
    for (int k = 0; k < c->prm.n_pd_iters; ++k) {
        kt.begin(DC_KT_LOCAL);
        launch_local(dm, P, xin, c->v, c->c1, c->c2, c->bu, s);
        kt.end(DC_KT_LOCAL);
        kt.begin(DC_KT_GATHER);
        launch_gather_rhs(dm, P, vin, c->c1, c->c2, c->bu, r.f, c->b, s);
        kt.end(DC_KT_GATHER);
        if (P.mass_split) {   // global step of the mass splitting (DC_COMPLIANCE_MASS)
            kt.begin(DC_KT_SOLVE_BWD);
            launch_mass_solve(dm, P, c->b, c->v, r.contact, r.nb, cc, r.f, r.case_, s);
            kt.end(DC_KT_SOLVE_BWD);
            continue;
        }
        kt.begin(DC_KT_SWEEPS);
        const bool fused = launch_solve_sweeps(dm, P, c->b, c->y, c->v, 1, r.contact, r.nb, cc, r.f, r.case_,
                                               nullptr, s);
        kt.end(DC_KT_SWEEPS);
        if (fused) continue;
        kt.begin(DC_KT_SOLVE_FWD);
        launch_solve_fwd(dm, c->b, c->y, s);
        kt.end(DC_KT_SOLVE_FWD);
        kt.begin(DC_KT_SOLVE_BWD);
        launch_solve_bwd(dm, P, c->y, c->v, 1, r.contact, r.nb, cc, r.f, r.case_, nullptr, s);
        kt.end(DC_KT_SOLVE_BWD);
    }
    launch_finalize(dm, P, xin, c->v, xout, c->counters + 4, s);
    if (vout != c->v) cudaMemcpyAsync(vout, c->v, sizeof(d4) * dm.m, cudaMemcpyDeviceToDevice, s);
    if (step >= 0 && c->d_inst_steps)
        launch_freeze(dm, P, c->d_inst_steps, step, step_base, xin, vin, xout, vout, r.contact, s);
    if (count) launch_count_cases(r.contact, r.case_, dm.m_free, c->counters, s);
}

namespace {

bool graphs_usable(const dc_ctx* c) {
    // the legacy and per-thread default streams cannot be captured
    return c->use_graphs && c->kt.cls == 0 && c->stream != nullptr && c->stream != cudaStreamLegacy &&
           c->stream != cudaStreamPerThread;
}

// Runs body() directly, or as a CUDA graph captured on first use for (ka, kb)
// in the current graph epoch and replayed afterwards.
template <class F>
dc_status run_graph(dc_ctx* c, GraphCache& gc, int ka, int kb, F body) {
    if (!graphs_usable(c)) {
        body();
        return DC_OK;
    }
    if (!gc.exec || gc.ka != ka || gc.kb != kb || gc.epoch != c->graph_epoch) {
        if (gc.exec) cudaGraphExecDestroy(gc.exec);
        gc.exec = nullptr;
        cudaGraph_t g = nullptr;
        const long long l0 = dc_launch_count();
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        body();
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        gc.launches = dc_launch_count() - l0;
        dc_add_launches(-gc.launches);   // counted when the graph is launched
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            c->err = std::string("CUDA graph capture failed: ") + cudaGetErrorString(e);
            return DC_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&gc.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            gc.exec = nullptr;
            c->err = std::string("CUDA graph instantiation failed: ") + cudaGetErrorString(e);
            return DC_ERR_CUDA;
        }
        gc.ka = ka;
        gc.kb = kb;
        gc.epoch = c->graph_epoch;
    }
    CK(cudaGraphLaunch(gc.exec, c->stream));
    dc_add_launches(gc.launches);
    c->graph_replays++;
    return DC_OK;
}

}  // namespace

dc_status rollout_steps(dc_ctx* c, int n_steps, int k) {
    const int m = c->hm.m;
    return run_graph(c, c->g_roll, n_steps, k, [&]() {
        d4 *cx = c->ck, *cv = c->ck + m;
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
            run_step(c, cx, cv, nx, nv, k == 1 ? c->rec_all[s] : c->scratch, true, s);
            cx = nx;
            cv = nv;
        }
        // the final state in xa / va for the caller (no copy when it is there already)
        if (cx != c->xa) cudaMemcpyAsync(c->xa, cx, sizeof(d4) * m, cudaMemcpyDeviceToDevice, c->stream);
        if (cv != c->va) cudaMemcpyAsync(c->va, cv, sizeof(d4) * m, cudaMemcpyDeviceToDevice, c->stream);
    });
}

dc_status ensure_checkpoints(dc_ctx* c, int n_ck) {
    if (n_ck <= c->ck_cap) return DC_OK;
    free_pool(c, c->ck_allocs);
    RET(dalloc(c, c->ck_allocs, &c->ck, (size_t)n_ck * 2 * c->hm.m));
    c->ck_cap = n_ck;
    c->graph_epoch++;
    return DC_OK;
}

dc_status ensure_records(dc_ctx* c, int n_steps) {
    if (n_steps <= c->rec_cap) return DC_OK;
    free_pool(c, c->rec_allocs);
    c->rec_all.assign(n_steps, StepRec{});
    for (int i = 0; i < n_steps; ++i) RET(alloc_rec(c, c->rec_allocs, c->rec_all[i]));
    c->rec_cap = n_steps;
    c->graph_epoch++;
    return DC_OK;
}

dc_status ensure_segment(dc_ctx* c, int k) {
    if (k <= c->seg_cap) return DC_OK;
    free_pool(c, c->seg_allocs);
    c->seg_rec.assign(k, StepRec{});
    RET(dalloc(c, c->seg_allocs, &c->segX, (size_t)(k + 1) * c->hm.m));
    RET(dalloc(c, c->seg_allocs, &c->segV, (size_t)(k + 1) * c->hm.m));
    for (int i = 0; i < k; ++i) RET(alloc_rec(c, c->seg_allocs, c->seg_rec[i]));
    c->seg_cap = k;
    c->graph_epoch++;
    return DC_OK;
}

dc_status recompute_segment(dc_ctx* c, int seg, int s0, int s1) {
    const int m = c->hm.m;
    cudaStream_t s = c->stream;
    const d4* ckx = c->ck + (size_t)seg * 2 * m;
    CK(cudaMemcpyAsync(c->segX, ckx, sizeof(d4) * m, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c->segV, ckx + m, sizeof(d4) * m, cudaMemcpyDeviceToDevice, s));
    const int n = s1 - s0;
    GraphCache& gc = c->g_seg[n == c->ck_every ? 0 : 1];
    // the segment's first step, read by the per-instance freeze inside the graph
    const int* base = c->d_inst_steps ? c->d_inst_steps + c->B : nullptr;
    if (base) launch_set_int(c->d_inst_steps + c->B, s0, s);
    return run_graph(c, gc, n, 0, [&]() {
        for (int q = 0; q < n; ++q)
            run_step(c, c->segX + (size_t)q * m, c->segV + (size_t)q * m, c->segX + (size_t)(q + 1) * m,
                     c->segV + (size_t)(q + 1) * m, c->seg_rec[q], false, base ? q : s0 + q, base);
    });
}

dc_status ensure_adjoint(dc_ctx* c) {
    int mr = std::max(1, std::min(256, c->prm.adj_restart));
    if (c->V && mr <= c->adj_restart_cap) return DC_OK;
    free_pool(c, c->adj_allocs);
    const int m = c->hm.m, mf = c->hm.m_free, T = c->hm.T, B = c->B;
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
        RET(dalloc(c, P, &a.tav, 4 * (size_t)T));
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
    RET(dalloc(c, P, &c->dcoef, (size_t)(mr + 1) * B));
    RET(dalloc(c, P, &c->dcoef2, (size_t)(mr + 1) * B));
    RET(dalloc(c, P, &c->dnorm, B));
    RET(dalloc(c, P, &c->dscale, B));
    RET(dalloc(c, P, &c->partial, (size_t)(mr + 1) * c->sg.nchunk));
    RET(dalloc(c, P, &c->dparam_acc, 4 * (size_t)B));
    RET(dalloc(c, P, &c->dparam_part, (size_t)c->sg.npchunk));
    if (B > 1 && c->prm.adj_precond == 0) {
        RET(dalloc(c, P, &c->d_act_sn, (size_t)std::max(c->fr.S, 1)));
        RET(dalloc(c, P, &c->d_act_ch, (size_t)std::max(c->sg.nchunk, 1)));
        if (c->h_act_sn) cudaFreeHost(c->h_act_sn);
        if (c->h_act_ch) cudaFreeHost(c->h_act_ch);
        c->h_act_sn = c->h_act_ch = nullptr;
        CK(cudaMallocHost(&c->h_act_sn, sizeof(int) * (size_t)std::max(c->fr.S, 1)));
        CK(cudaMallocHost(&c->h_act_ch, sizeof(int) * (size_t)std::max(c->sg.nchunk, 1)));
    }
    const size_t need = 3 * (size_t)(mr + 1) * B + 4 * (size_t)B + 64;
    if (need > c->hpin_cap) {
        if (c->hpin && !c->hpin_external) cudaFreeHost(c->hpin);
        c->hpin_external = false;
        c->hpin = nullptr;
        c->hpin_cap = 0;
        CK(cudaMallocHost(&c->hpin, need * sizeof(double)));
        c->hpin_cap = need;
    }
    c->adj_restart_cap = mr;
    return DC_OK;
}

namespace {

inline d4* vcol(double* base, int j, int m) { return reinterpret_cast<d4*>(base + (size_t)j * 4 * m); }

// Preconditioner K(w) -> out.
void precond(dc_ctx* c, const AdjDev& ad, const d4* w, d4* out) {
    cudaStream_t s = c->stream;
    const DevMesh& dm = c->dm;
    if (c->prm.adj_precond == 0) {
        frontal_precond(ad, c->fdv, c->fr.lvl_ptr.data(), c->nlev, c->lvl_maxf.data(), dm.m_free, w, out, s,
                        &c->kt, c->act_on ? c->d_act_sn : nullptr, c->act_ptr.data(),
                        c->act_on ? c->d_act_sn : nullptr, c->n_act_tq);
        return;
    }
    // node-block inverse, projected P^-1, node-block inverse
    adj_dplus(dm, ad, nullptr, w, c->x1, s);
    adj_apply_H(dm, ad, 1, c->x1, w, c->r1, s);
    adj_solve_project(dm, ad, c->r1, c->ytmp, c->x1, c->x2, s);
    adj_apply_H(dm, ad, 1, c->x2, w, c->r2, s);
    adj_dplus(dm, ad, c->x2, c->r2, out, s);
}

// The fallback's preconditioner: K w (the per-step one), then one sweep of the
// constrained node-block inverse D+ of H on what K left, out = K w + D+ (w - Pi_B H K w).
void precond_fallback(dc_ctx* c, const AdjDev& ad, const d4* w, d4* out) {
    precond(c, ad, w, out);
    adj_apply_H(c->dm, ad, 1, out, w, c->r2, c->stream);
    adj_dplus(c->dm, ad, out, c->r2, out, c->stream);
}

// Compacted front and chunk lists of the instances with gs[i].act (batches only).
dc_status build_active_lists(dc_ctx* c) {
    const int B = c->B, nl = c->nlev;
    c->act_ptr.assign(nl + 1, 0);
    int pos = 0, cnt = 0;
    for (int i = 0; i < B; ++i) cnt += c->gs[i].act;
    if (c->fdv.tree) {
        for (int s : c->tq_h)
            if (c->gs[c->sn_inst_h[s]].act) c->h_act_sn[pos++] = s;
        c->n_act_tq = pos;
    } else {
        for (int l = 0; l < nl; ++l) {
            c->act_ptr[l] = pos;
            const int* P = c->lvl_inst_ptr.data() + (size_t)l * (B + 1);
            for (int i = 0; i < B; ++i)
                if (c->gs[i].act)
                    for (int q = P[i]; q < P[i + 1]; ++q) c->h_act_sn[pos++] = c->fr.lvl_sn[q];
        }
        c->act_ptr[nl] = pos;
    }
    if (pos > 0)
        CK(cudaMemcpyAsync(c->d_act_sn, c->h_act_sn, sizeof(int) * pos, cudaMemcpyHostToDevice, c->stream));
    int nch = 0;
    for (int i = 0; i < B; ++i)
        if (c->gs[i].act)
            for (int q = c->h_cptr[i]; q < c->h_cptr[i + 1]; ++q) c->h_act_ch[nch++] = q;
    c->n_act_ch = nch;
    if (nch > 0)
        CK(cudaMemcpyAsync(c->d_act_ch, c->h_act_ch, sizeof(int) * nch, cudaMemcpyHostToDevice, c->stream));
    c->act_on = true;
    c->act_built = cnt;
    return DC_OK;
}

// Per-instance |a|^2-style dot products a . b into out[0 .. B).
dc_status bdot_host(dc_ctx* c, const double* a, const double* b, std::vector<double>& out) {
    c->kt.begin(DC_KT_KRYLOV);
    adj_bdot(c->sg, a, 0, 1, b, c->partial, c->dnorm, c->stream);
    c->kt.end(DC_KT_KRYLOV);
    CK(cudaMemcpyAsync(c->hpin, c->dnorm, sizeof(double) * c->B, cudaMemcpyDeviceToHost, c->stream));
    CK(ctx_sync(c, c->stream));
    out.assign(c->hpin, c->hpin + c->B);
    return DC_OK;
}

dc_status upload_scale(dc_ctx* c, const std::vector<double>& sc) {
    double* h = c->hpin + 3 * (size_t)(c->adj_restart_cap + 1) * c->B;
    // the previous upload from this buffer must have been consumed
    CK(ctx_sync(c, c->stream));
    std::memcpy(h, sc.data(), sizeof(double) * c->B);
    CK(cudaMemcpyAsync(c->dscale, h, sizeof(double) * c->B, cudaMemcpyHostToDevice, c->stream));
    return DC_OK;
}

}  // namespace

// Flexible GMRES for Pi_B H z = rhs with z in null(C^T), run for every instance
// of the context in lockstep: one Arnoldi step is one set of launches over all
// instances, with per-instance dot products, Hessenberg columns, Givens
// rotations, convergence tests and restarts.  An instance that has converged
// (or stagnated, or reached the cap) is frozen with zero Krylov vectors, so its
// iterates are exactly those of a run on its own.  iters[i] and rel[i] receive
// each instance's iteration count and final relative residual (to |rhs_i|).
//
// The fallback pass (fallback = true) runs only the instances with sel[i] set,
// continuing from their current z (its first residual is rhs - Pi_B H z), as
// GMRES(30) with the stronger preconditioner precond_fallback, an iteration
// budget of max(adj_max_iters, 300), and a restart cycle counted as stagnated
// only when it fails to cut the residual by 10% (the first pass stops at 50%,
// which keeps lockstep batches short; the short restart makes a fallback that
// cannot get further stop after 30 iterations).
dc_status gmres(dc_ctx* c, std::vector<int>& iters, std::vector<double>& rel, bool fallback = false,
                const std::vector<char>* sel = nullptr) {
    cudaStream_t s = c->stream;
    const int m = c->hm.m, B = c->B;
    const long ldv = 4L * m;
    const int mr_cap = std::max(1, std::min(256, c->prm.adj_restart));
    const int mr = fallback ? std::min(30, mr_cap) : mr_cap;
    const int maxit = fallback ? std::max(c->prm.adj_max_iters, 300) : std::max(1, c->prm.adj_max_iters);
    const double tol = c->prm.adj_tol;
    const double stagnate = fallback ? 0.9 : 0.5;
    double* zz = reinterpret_cast<double*>(c->z);
    double* rr = reinterpret_cast<double*>(c->r1);
    if (!fallback) CK(cudaMemsetAsync(c->z, 0, sizeof(d4) * m, s));
    std::vector<double> nrm;
    RET(bdot_host(c, reinterpret_cast<double*>(c->rhs), reinterpret_cast<double*>(c->rhs), nrm));
    std::vector<GState>& gs = c->gs;
    gs.assign(B, GState());
    bool any = false;
    for (int i = 0; i < B; ++i) {
        gs[i].beta0 = std::sqrt(nrm[i]);
        if (!std::isfinite(gs[i].beta0)) {
            c->err = "non-finite adjoint right-hand side (instance " + std::to_string(i) + ")";
            return DC_ERR_NONFINITE;
        }
        gs[i].fin = !(gs[i].beta0 > 0.0) || (sel && !(*sel)[i]);
        any |= !gs[i].fin;
    }
    iters.assign(B, 0);
    rel.assign(B, 0.0);
    if (!any) return DC_OK;
    // per instance: Hessenberg columns (column j has j + 2 entries), rotations, rhs
    std::vector<std::vector<double>> Hc(B), cs(B), sn(B), gg(B);
    std::vector<char> done(B, 0);
    std::vector<double> sc(B, 0.0), yv;
    if (fallback) {   // residual of the current iterate
        c->kt.begin(DC_KT_APPLYH);
        adj_apply_H(c->dm, c->ad, 1, c->z, c->rhs, c->r1, s);
        c->kt.end(DC_KT_APPLYH);
    } else {
        CK(cudaMemcpyAsync(c->r1, c->rhs, sizeof(d4) * m, cudaMemcpyDeviceToDevice, s));
    }
    const bool debug = std::getenv("DC_DEBUG_GMRES") != nullptr;
    const long long lock0 = c->adj_batch_iters;
    for (int cycle = 0;; ++cycle) {
        RET(bdot_host(c, rr, rr, nrm));
        bool active = false;
        for (int i = 0; i < B; ++i) {
            GState& g = gs[i];
            g.act = false;
            if (g.fin) continue;
            const double beta = std::sqrt(nrm[i]);
            g.res = beta;
            if (debug && i == 0)
                std::fprintf(stderr, "[dc gmres] cycle %d iters %d true rel residual %.3e\n", cycle, g.total,
                             beta / g.beta0);
            // converged, capped, or a restart that did not halve the true residual
            // (the rounding floor, about eps * cond(H), has been reached)
            if (beta <= tol * g.beta0 || g.total >= maxit || (cycle > 0 && beta > stagnate * g.prev)) {
                g.fin = true;
                continue;
            }
            g.prev = beta;
            g.act = true;
            g.used = 0;
            active = true;
            Hc[i].clear();
            cs[i].assign(mr, 0.0);
            sn[i].assign(mr, 0.0);
            gg[i].assign(mr + 1, 0.0);
            gg[i][0] = beta;
            done[i] = 0;
        }
        if (!active) break;
        if (c->h_act_sn) RET(build_active_lists(c));
        for (int i = 0; i < B; ++i) sc[i] = gs[i].act ? 1.0 / gs[i].res : 0.0;
        RET(upload_scale(c, sc));
        // chunk list of the active instances (batches), else all chunks
        const int* cl = c->h_act_sn ? c->d_act_ch : nullptr;
        c->kt.begin(DC_KT_KRYLOV);
        adj_bscale(c->sg, rr, c->dscale, c->V, s, cl, c->n_act_ch);
        c->kt.end(DC_KT_KRYLOV);
        int jmax = 0;
        // inside the Arnoldi loop the instances whose scale is 0 (finished) are
        // skipped by every kernel
        AdjDev adm = c->ad;
        const double* mask = c->dscale;
        adm.mask = mask;
        for (int j = 0; j < mr; ++j) {
            d4* vj = vcol(c->V, j, m);
            d4* zj = vcol(c->Zb, j, m);
            if (fallback)
                precond_fallback(c, adm, vj, zj);
            else
                precond(c, adm, vj, zj);
            c->kt.begin(DC_KT_APPLYH);
            adj_apply_H(c->dm, adm, 0, zj, nullptr, c->wv, s);
            c->kt.end(DC_KT_APPLYH);
            double* w = reinterpret_cast<double*>(c->wv);
            // classical Gram-Schmidt, twice
            c->kt.begin(DC_KT_KRYLOV);
            const int ncl = c->n_act_ch;
            adj_bdot(c->sg, c->V, ldv, j + 1, w, c->partial, c->dcoef, s, mask, cl, ncl);
            adj_bvupdate(c->sg, c->V, ldv, j + 1, c->dcoef, w, -1.0, s, mask, cl, ncl);
            adj_bdot(c->sg, c->V, ldv, j + 1, w, c->partial, c->dcoef2, s, mask, cl, ncl);
            adj_bvupdate(c->sg, c->V, ldv, j + 1, c->dcoef2, w, -1.0, s, mask, cl, ncl);
            adj_bdot(c->sg, w, 0, 1, w, c->partial, c->dnorm, s, mask, cl, ncl);
            c->kt.end(DC_KT_KRYLOV);
            double* h1 = c->hpin;
            double* h2 = c->hpin + (size_t)(mr + 1) * B;
            double* hn_all = c->hpin + 2 * (size_t)(mr + 1) * B;
            CK(cudaMemcpyAsync(h1, c->dcoef, sizeof(double) * (j + 1) * B, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(h2, c->dcoef2, sizeof(double) * (j + 1) * B, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(hn_all, c->dnorm, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
            CK(ctx_sync(c, s));
            bool still = false;
            for (int i = 0; i < B; ++i) {
                GState& g = gs[i];
                sc[i] = 0.0;
                if (!g.act) continue;
                std::vector<double>& H = Hc[i];
                const size_t o = H.size();
                H.resize(o + j + 2);
                double* hc = H.data() + o;
                for (int k = 0; k <= j; ++k) hc[k] = h1[(size_t)k * B + i] + h2[(size_t)k * B + i];
                const double hn = std::sqrt(std::max(hn_all[i], 0.0));
                hc[j + 1] = hn;
                if (!std::isfinite(hn)) {
                    c->err = "non-finite value in the adjoint iteration (instance " + std::to_string(i) + ")";
                    return DC_ERR_NONFINITE;
                }
                for (int k = 0; k < j; ++k) {
                    double t = cs[i][k] * hc[k] + sn[i][k] * hc[k + 1];
                    hc[k + 1] = -sn[i][k] * hc[k] + cs[i][k] * hc[k + 1];
                    hc[k] = t;
                }
                const double den = std::hypot(hc[j], hc[j + 1]);
                cs[i][j] = den > 0 ? hc[j] / den : 1.0;
                sn[i][j] = den > 0 ? hc[j + 1] / den : 0.0;
                hc[j] = den;
                hc[j + 1] = 0.0;
                gg[i][j + 1] = -sn[i][j] * gg[i][j];
                gg[i][j] = cs[i][j] * gg[i][j];
                g.total++;
                g.used = j + 1;
                g.res = std::fabs(gg[i][j + 1]);
                if (g.res <= tol * g.beta0 || g.total >= maxit || hn == 0.0) {
                    g.act = false;
                    done[i] = 1;
                } else {
                    sc[i] = 1.0 / hn;
                    still = true;
                }
            }
            jmax = j + 1;
            c->adj_batch_iters++;
            if (!still) break;
            if (c->h_act_sn) {
                int cnt = 0;
                for (int i = 0; i < B; ++i) cnt += gs[i].act;
                if (4 * cnt <= 3 * c->act_built) RET(build_active_lists(c));
            }
            RET(upload_scale(c, sc));
            c->kt.begin(DC_KT_KRYLOV);
            adj_bscale(c->sg, w, c->dscale, reinterpret_cast<double*>(vcol(c->V, j + 1, m)), s, cl, c->n_act_ch);
            c->kt.end(DC_KT_KRYLOV);
        }
        // z += sum_j Zb_j y_j per instance (columns past an instance's own count are 0)
        double* hy = c->hpin;
        CK(ctx_sync(c, s));
        std::memset(hy, 0, sizeof(double) * (size_t)jmax * B);
        for (int i = 0; i < B; ++i) {
            const GState& g = gs[i];
            if (g.fin || g.used == 0) continue;
            const int used = g.used;
            yv.assign(used, 0.0);
            const double* H = Hc[i].data();
            auto Hat = [&](int k, int r) { return H[(size_t)k * (k + 3) / 2 + r]; };   // column k starts at k(k+3)/2
            for (int r = used - 1; r >= 0; --r) {
                double t = gg[i][r];
                for (int k = r + 1; k < used; ++k) t -= Hat(k, r) * yv[k];
                yv[r] = t / Hat(r, r);
            }
            for (int k = 0; k < used; ++k) hy[(size_t)k * B + i] = yv[k];
        }
        CK(cudaMemcpyAsync(c->dcoef, hy, sizeof(double) * (size_t)jmax * B, cudaMemcpyHostToDevice, s));
        c->kt.begin(DC_KT_KRYLOV);
        adj_bvupdate(c->sg, c->Zb, ldv, jmax, c->dcoef, zz, 1.0, s);
        c->kt.end(DC_KT_KRYLOV);
        // true residual r = rhs - Pi_B H z
        c->kt.begin(DC_KT_APPLYH);
        adj_apply_H(c->dm, c->ad, 1, c->z, c->rhs, c->r1, s);
        c->kt.end(DC_KT_APPLYH);
        bool capped = false;
        for (int i = 0; i < B; ++i) capped |= !gs[i].fin && done[i] && gs[i].total >= maxit;
        if (capped) {
            RET(bdot_host(c, rr, rr, nrm));
            for (int i = 0; i < B; ++i)
                if (!gs[i].fin && done[i] && gs[i].total >= maxit) {
                    gs[i].res = std::sqrt(nrm[i]);
                    gs[i].fin = true;
                }
        }
        for (int i = 0; i < B; ++i) gs[i].used = 0;
    }
    c->act_on = false;
    if (debug && std::getenv("DC_DEBUG_GMRES")[0] == '2') {
        int mx = 0, arg = 0, over8 = 0;
        for (int i = 0; i < B; ++i) {
            if (gs[i].total > mx) mx = gs[i].total, arg = i;
            over8 += gs[i].total > 8;
        }
        const double r = gs[arg].beta0 > 0.0 ? gs[arg].res / gs[arg].beta0 : 0.0;
        std::fprintf(stderr,
                     "[dc gmres] step: %lld lockstep iterations, largest instance total %d (instance %d, rel "
                     "residual %.3e), %d instances above 8\n",
                     c->adj_batch_iters - lock0, mx, arg, r, over8);
    }
    for (int i = 0; i < B; ++i) {
        iters[i] = gs[i].total;
        rel[i] = gs[i].beta0 > 0.0 ? gs[i].res / gs[i].beta0 : 0.0;
        if (debug && !(rel[i] <= tol))
            std::fprintf(stderr, "[dc gmres] instance %d stopped at %d iterations, rel residual %.3e (beta0 %.3e)\n",
                         i, iters[i], rel[i], gs[i].beta0);
    }
    return DC_OK;
}

// Per-step adjoint data of step q into slot k: the element linearisation, node
// types and (with the multifrontal preconditioner) the factorised fronts.  Runs on
// stream2 so that it overlaps the GMRES of the step after q.
void prepare_step(dc_ctx* c, const StepRec& r, const d4* x1, const d4* v1, int k, cudaStream_t s) {
    AdjDev& ad = c->ads[k];
    ad.h = c->prm.h;
    ad.mu = c->dp.node_mu;
    ad.node_inst = c->dp.node_inst;
    ad.mask = nullptr;
    ad.contact = r.contact;
    ad.case_ = r.case_;
    ad.nb = r.nb;
    ad.f = r.f;
    KTimer* kt = s == c->stream ? &c->kt : &c->kt2;
    kt->begin(DC_KT_ASSEMBLE);
    adj_setup(c->dm, ad, x1, v1, s);
    kt->end(DC_KT_ASSEMBLE);
    if (c->prm.adj_precond == 0) {
        frontal_factorize(c->dm, ad, c->fds[k], c->fr.lvl_ptr.data(), c->nlev, c->lvl_maxf.data(), c->lvl_maxp.data(), s,
                          s == c->stream ? &c->kt : &c->kt2);
        c->n_factorisations++;
    }
}

// One adjoint step from slot k: (gx, gv) at n+1 -> (gx2, gv2) at n, parameter
// terms into dparam_acc.
dc_status adjoint_step(dc_ctx* c, const d4* x_n, const d4* x1, const d4* v1, int k, bool& noncv, int step) {
    cudaStream_t s = c->stream;
    c->ad = c->ads[k];
    c->fdv = c->fds[k];
    AdjDev& ad = c->ad;
    adj_rhs(c->dm, ad, c->gx, c->gv, c->g, c->rhs, s);
    std::vector<int> it;
    std::vector<double> rel;
    // instances past their own last step take no part (their adjoint passes through)
    std::vector<char> live;
    if (c->d_inst_steps) {
        live.assign(c->B, 1);
        for (int i = 0; i < c->B; ++i) live[i] = c->inst_steps[i] > step;
    }
    RET(gmres(c, it, rel, false, live.empty() ? nullptr : &live));
    if (c->prm.adj_fallback) {
        // instances that hit the iteration cap, or stopped more than 100 x adj_tol
        // above it: a second pass from their iterate.  A restart cycle that fails
        // to halve the residual close to adj_tol has met the rounding floor of the
        // FP64 operator (about eps cond(H)), which no preconditioner moves; those
        // steps are accepted and counted as non-converged.
        std::vector<char> sel(c->B, 0);
        bool any = false;
        const int maxit = std::max(1, c->prm.adj_max_iters);
        for (int i = 0; i < c->B; ++i)
            if (!(rel[i] <= c->prm.adj_tol * 1.0000001) && (it[i] >= maxit || !(rel[i] <= 100.0 * c->prm.adj_tol)))
                sel[i] = 1, any = true;
        if (any) {
            std::vector<int> it2;
            std::vector<double> rel2;
            RET(gmres(c, it2, rel2, true, &sel));
            for (int i = 0; i < c->B; ++i)
                if (sel[i]) {
                    c->adj_fallbacks++;
                    c->adj_fallback_iters += it2[i];
                    it[i] += it2[i];
                    rel[i] = rel2[i];
                }
        }
    }
    if ((int)c->inst_noncv.size() != c->B) c->inst_noncv.assign(c->B, 0);
    for (int i = 0; i < c->B; ++i) {
        c->adj_steps++;
        c->adj_iters += it[i];
        c->adj_max_seen = std::max<long long>(c->adj_max_seen, it[i]);
        if (!(rel[i] <= c->prm.adj_tol * 1.0000001)) {
            c->adj_noncv++;
            c->inst_noncv[i]++;
            noncv = true;
        }
    }
    c->adj_last_res = *std::max_element(rel.begin(), rel.end());
    adj_apply_H(c->dm, ad, 3, c->z, nullptr, c->E, s);
    adj_apply_H(c->dm, ad, 2, c->z, c->g, c->resid, s);
    adj_outputs(c->dm, ad, c->dp, c->z, c->E, c->resid, x_n, v1, c->gx, c->gx2, c->gv2, s);
    if (c->d_inst_steps) launch_pass_adjoint(c->dm, c->dp, c->d_inst_steps, step, c->gv, c->gv2, s);
    adj_params(c->dm, ad, c->sg, c->z, x1, c->dparam_part, c->dparam_acc, s);
    CK(cudaEventRecord(c->ev_free[k], s));
    std::swap(c->gx, c->gx2);
    std::swap(c->gv, c->gv2);
    return DC_OK;
}

// Block-size autotuner: times the local-step, gather, per-node and adjoint
// element kernels at 64..512 threads per block on this context's mesh (rest
// state, zero velocity) and keeps the fastest of each.  The launch shape of
// these kernels changes no result (one thread per element or node).
dc_status autotune(dc_ctx* c) {
    RET(ensure_adjoint(c));
    cudaStream_t s = c->stream;
    const int m = c->hm.m;
    {
        std::vector<d4> h(m);
        for (int i = 0; i < m; ++i) h[i] = d4{c->hm.rest[3 * i], c->hm.rest[3 * i + 1], c->hm.rest[3 * i + 2], 0.0};
        CK(cudaMemcpyAsync(c->xa, h.data(), sizeof(d4) * m, cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(c->va, 0, sizeof(d4) * m, s));
        CK(cudaMemsetAsync(c->v, 0, sizeof(d4) * m, s));
        CK(cudaMemsetAsync(c->scratch.f, 0, sizeof(d4) * c->hm.m_free, s));
        CK(ctx_sync(c, s));
    }
    AdjDev ad = c->ads[0];
    ad.h = c->prm.h;
    ad.mu = c->dp.node_mu;
    ad.node_inst = c->dp.node_inst;
    ad.mask = nullptr;
    ad.contact = c->scratch.contact;
    ad.case_ = c->scratch.case_;
    ad.nb = c->scratch.nb;
    ad.f = c->scratch.f;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int cand[] = {64, 128, 256, 512};
    auto time_it = [&](auto launch) -> float {
        for (int w = 0; w < 2; ++w) launch();
        cudaEventRecord(e0, s);
        for (int r = 0; r < 8; ++r) launch();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    auto pick = [&](int* field, auto launch) {
        float best = 1e30f;
        int arg = *field;
        for (int b : cand) {
            *field = b;
            float t = time_it(launch);
            if (t < best) {
                best = t;
                arg = b;
            }
        }
        *field = arg;
    };
    DevMesh& dm = c->dm;
    const DevParams& P = c->dp;
    pick(&dm.bs_local, [&]() { launch_local(dm, P, c->xa, c->v, c->c1, c->c2, c->bu, s); });
    pick(&dm.bs_gather, [&]() { launch_gather_rhs(dm, P, c->va, c->c1, c->c2, c->bu, c->scratch.f, c->b, s); });
    pick(&dm.bs_node, [&]() {
        launch_detect(dm, P, c->xa, c->va, c->scratch.contact, c->scratch.nb, c->scratch.f, c->ind, s);
        launch_finalize(dm, P, c->xa, c->v, c->xb, c->counters + 4, s);
    });
    pick(&dm.bs_elem, [&]() { adj_apply_H(dm, ad, 0, c->v, nullptr, c->wv, s); });
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(ctx_sync(c, s));
    CK(cudaGetLastError());
    c->graph_epoch++;
    return DC_OK;
}
