// Context setup in two halves: host preparation (merging the instances' meshes,
// factorising every instance's PD matrix, building the adjoint fronts and the
// per-instance tables) and the device upload of its results.  A plain context
// runs both back to back; the request server prepares on host threads and
// uploads on the stream of the slot that runs the request.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <string>
#include <thread>

#include "dc_ctx.h"

namespace {

constexpr int CHUNK_D = 512;    // doubles per reduction chunk of the Krylov vectors (128 nodes)
constexpr int CHUNK_E = 1024;   // elements per chunk of the parameter-gradient terms

bool finite_params(const dc_params& p) {
    const double v[] = {p.k_stretch, p.k_bend, p.density, p.mu, p.h, p.gravity[0], p.gravity[1], p.gravity[2],
                        p.contact_margin, p.adj_tol};
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

// Validates q and normalises its obstacles (unit plane normals).  "" or an error.
std::string normalise_params(dc_params& q) {
    if (!finite_params(q) || !(q.h > 0) || q.k_stretch < 0 || q.k_bend < 0 || !(q.density > 0) || q.mu < 0 ||
        q.n_pd_iters < 0 || q.n_obstacles < 0 || q.n_obstacles > DC_MAX_OBSTACLES || q.checkpoint_every < 1 ||
        q.adj_max_iters < 1 || q.adj_restart < 1 || !(q.adj_tol > 0) || q.adj_precond < 0 || q.adj_precond > 1 ||
        q.global_solver < 0 || q.global_solver > 1 || q.contact_compliance < DC_COMPLIANCE_ROWSUM ||
        q.contact_compliance > DC_COMPLIANCE_MASS || q.adj_fallback < 0 || q.adj_fallback > 1 ||
        q.factor_on_gpu < 0 || q.factor_on_gpu > 1)
        return "invalid or non-finite parameter";
    if (q.factor_on_gpu == 1 && q.global_solver != 1)
        return "factor_on_gpu needs global_solver 1 (the GPU factor is written as supernodal panels)";
    if (q.factor_on_gpu == 1 && q.contact_compliance == DC_COMPLIANCE_DIAG_PINV)
        return "DC_COMPLIANCE_DIAG_PINV needs the host factor (factor_on_gpu 0)";
    if (q.adj_precond == 1 && q.global_solver != 0)
        return "adj_precond 1 needs global_solver 0 (it projects with the explicit inverse rows)";
    for (int o = 0; o < q.n_obstacles; ++o) {
        dc_obstacle& ob = q.obstacles[o];
        for (int k = 0; k < 7; ++k)
            if (!std::isfinite(ob.p[k])) return "non-finite obstacle";
        if (ob.kind == DC_PLANE) {
            double nn = std::sqrt(ob.p[0] * ob.p[0] + ob.p[1] * ob.p[1] + ob.p[2] * ob.p[2]);
            if (!(nn > 0)) return "zero plane normal";
            for (int k = 0; k < 3; ++k) ob.p[k] /= nn;
            ob.p[3] /= nn;
        } else if (ob.kind == DC_SPHERE) {
            if (!(ob.p[3] > 0)) return "sphere radius must be positive";
        } else if (ob.kind == DC_CAPSULE) {
            double L = std::fabs(ob.p[3] - ob.p[0]) + std::fabs(ob.p[4] - ob.p[1]) + std::fabs(ob.p[5] - ob.p[2]);
            if (!(ob.p[6] > 0) || !(L > 0)) return "bad capsule";
        } else if (ob.kind == DC_MESH) {
            if (!(ob.p[0] >= 0) || ob.p[0] != std::floor(ob.p[0])) return "bad obstacle mesh id";
        } else {
            return "unknown obstacle kind";
        }
    }
    return "";
}

}  // namespace

// The fields every instance of a batch must share.
bool dc_same_batch_fields(const dc_params& a, const dc_params& b) {
    return a.h == b.h && a.gravity[0] == b.gravity[0] && a.gravity[1] == b.gravity[1] &&
           a.gravity[2] == b.gravity[2] && a.contact_margin == b.contact_margin && a.adj_tol == b.adj_tol &&
           a.n_pd_iters == b.n_pd_iters && a.adj_max_iters == b.adj_max_iters && a.adj_restart == b.adj_restart &&
           a.checkpoint_every == b.checkpoint_every && a.adj_precond == b.adj_precond &&
           a.global_solver == b.global_solver && a.contact_compliance == b.contact_compliance &&
           a.adj_fallback == b.adj_fallback && a.factor_on_gpu == b.factor_on_gpu;
}

namespace {

bool same_batch_fields(const dc_params& a, const dc_params& b) { return dc_same_batch_fields(a, b); }

template <class T>
size_t vbytes(const std::vector<T>& v) {
    return std::max<size_t>(v.size() * sizeof(T), 32);
}

}  // namespace

void dc_parallel_for(int n, const std::function<void(int)>& f) {
    int nt = (int)std::min<unsigned>((unsigned)std::max(n, 1), std::max(1u, std::thread::hardware_concurrency()));
    if (nt <= 1) {
        for (int i = 0; i < n; ++i) f(i);
        return;
    }
    std::atomic<int> next{0};
    std::vector<std::thread> th;
    th.reserve(nt);
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&]() {
            for (int i; (i = next.fetch_add(1)) < n;) f(i);
        });
    for (auto& t : th) t.join();
}

void prep_mesh_host(dc_ctx* c, MeshPrep& mp) {
    dc_merge_meshes(c->ihm, c->inst, c->hm);
    c->B = (int)c->ihm.size();
    const HostMesh& hm = c->hm;
    const int m = hm.m, T = hm.T, MF = hm.m_free, B = c->B;
    mp.tri4.resize(T);
    mp.G4.resize(T);
    for (int t = 0; t < T; ++t) {
        mp.tri4[t] = make_int4(hm.tri[3 * t], hm.tri[3 * t + 1], hm.tri[3 * t + 2], 0);
        mp.G4[t] = d4{hm.G[4 * t], hm.G[4 * t + 1], hm.G[4 * t + 2], hm.G[4 * t + 3]};
    }
    mp.qr.resize(m);
    for (int i = 0; i < m; ++i) mp.qr[i] = d4{hm.qrest[3 * i], hm.qrest[3 * i + 1], hm.qrest[3 * i + 2], 0.0};
    // node -> triangle incidences and transposed bending stencils (counting sort:
    // every list keeps ascending triangle / row order)
    auto& iptr = mp.iptr;
    auto& tbptr = mp.tbptr;
    iptr.assign(m + 1, 0);
    tbptr.assign(m + 1, 0);
    for (int t = 0; t < T; ++t)
        for (int a = 0; a < 3; ++a) iptr[hm.tri[3 * t + a] + 1]++;
    for (int i = 0; i < m; ++i) iptr[i + 1] += iptr[i];
    mp.iidx.assign(iptr[m], 0);
    std::vector<int> fill(iptr.begin(), iptr.end() - 1);
    for (int t = 0; t < T; ++t)
        for (int a = 0; a < 3; ++a) mp.iidx[fill[hm.tri[3 * t + a]]++] = 3 * t + a;
    for (int b = 0; b < m; ++b)
        for (int k = hm.bptr[b]; k < hm.bptr[b + 1]; ++k) tbptr[hm.bidx[k] + 1]++;
    for (int i = 0; i < m; ++i) tbptr[i + 1] += tbptr[i];
    mp.tbidx.assign(tbptr[m], 0);
    mp.tbval.assign(tbptr[m], 0.0);
    fill.assign(tbptr.begin(), tbptr.end() - 1);
    for (int b = 0; b < m; ++b)
        for (int k = hm.bptr[b]; k < hm.bptr[b + 1]; ++k) {
            int q = fill[hm.bidx[k]]++;
            mp.tbidx[q] = b;
            mp.tbval[q] = hm.bval[k];
        }
    // instance of every node; reduction chunks counted from each instance's start
    mp.node_inst.assign(m, 0);
    mp.cptr.assign(B + 1, 0);
    mp.pcptr.assign(3 * B + 1, 0);
    mp.chunks.clear();
    mp.pchunks.clear();
    for (int i = 0; i < B; ++i) {
        const InstInfo& in = c->inst[i];
        for (int l = 0; l < in.m; ++l) mp.node_inst[in.map(l, MF)] = i;
        for (int a = 4 * in.fo; a < 4 * (in.fo + in.mf); a += CHUNK_D)
            mp.chunks.push_back(make_int4(i, a, std::min(4 * (in.fo + in.mf), a + CHUNK_D), 0));
        mp.cptr[i + 1] = (int)mp.chunks.size();
        auto add = [&](int kind, int lo, int hi) {
            for (int a = lo; a < hi; a += CHUNK_E)
                mp.pchunks.push_back(make_int4(i, kind, a, std::min(hi, a + CHUNK_E)));
        };
        add(0, in.to, in.to + in.T);
        mp.pcptr[3 * i + 1] = (int)mp.pchunks.size();
        add(1, in.fo, in.fo + in.mf);
        add(1, MF + in.po, MF + in.po + (in.m - in.mf));
        mp.pcptr[3 * i + 2] = (int)mp.pchunks.size();
        add(2, in.fo, in.fo + in.mf);
        mp.pcptr[3 * i + 3] = (int)mp.pchunks.size();
    }
    if (mp.chunks.empty()) mp.chunks.push_back(make_int4(0, 0, 0, 0));   // keeps every launch non-empty
}

dc_status upload_mesh(dc_ctx* c, MeshPrep& mp) {
    const HostMesh& hm = c->hm;
    auto& P = c->mesh_allocs;
    int4* d_tri;
    d4 *d_G, *d_qr;
    double *d_area, *d_bval, *d_abar, *d_sb, *d_tbval;
    int *d_bptr, *d_bidx, *d_iptr, *d_iidx, *d_tbptr, *d_tbidx, *d_ninst, *d_cptr, *d_pcptr;
    int4 *d_chunks, *d_pchunks;
    dc_status s;
    if ((s = upload(c, P, &d_tri, mp.tri4)) || (s = upload(c, P, &d_G, mp.G4)) ||
        (s = upload(c, P, &d_area, hm.area)) || (s = upload(c, P, &d_bptr, hm.bptr)) ||
        (s = upload(c, P, &d_bidx, hm.bidx)) || (s = upload(c, P, &d_bval, hm.bval)) ||
        (s = upload(c, P, &d_abar, hm.abar)) || (s = upload(c, P, &d_sb, hm.sb)) || (s = upload(c, P, &d_qr, mp.qr)) ||
        (s = upload(c, P, &d_iptr, mp.iptr)) || (s = upload(c, P, &d_iidx, mp.iidx)) ||
        (s = upload(c, P, &d_tbptr, mp.tbptr)) || (s = upload(c, P, &d_tbidx, mp.tbidx)) ||
        (s = upload(c, P, &d_tbval, mp.tbval)) || (s = upload(c, P, &c->d_int2ext, hm.int2ext)) ||
        (s = upload(c, P, &d_ninst, mp.node_inst)) || (s = upload(c, P, &d_cptr, mp.cptr)) ||
        (s = upload(c, P, &d_pcptr, mp.pcptr)) || (s = upload(c, P, &d_chunks, mp.chunks)) ||
        (s = upload(c, P, &d_pchunks, mp.pchunks)))
        return s;
    const int m = hm.m, T = hm.T;
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
    dm.bs_local = dm.bs_gather = dm.bs_elem = dm.bs_node = 128;
    c->dp.node_inst = d_ninst;
    c->sg.B = c->B;
    c->sg.nchunk = (int)mp.chunks.size();
    c->sg.chunk = d_chunks;
    c->sg.cptr = d_cptr;
    c->sg.npchunk = (int)mp.pchunks.size();
    c->sg.pchunk = d_pchunks;
    c->sg.pcptr = d_pcptr;
    c->h_cptr = mp.cptr;
    // work buffers
    auto& W = c->work_allocs;
    d4** vecs[] = {&c->xa, &c->va, &c->xb, &c->vb, &c->v, &c->b, &c->y, &c->bu, &c->ind};
    for (d4** p : vecs) RET(dalloc(c, W, p, m));
    RET(dalloc(c, W, &c->c1, T));
    RET(dalloc(c, W, &c->c2, T));
    RET(dalloc(c, W, &c->cc, m));
    RET(dalloc(c, W, &c->stage, 3 * (size_t)m));
    RET(dalloc(c, W, &c->stage2, 3 * (size_t)m));
    RET(dalloc(c, W, &c->counters, 8));
    RET(alloc_rec(c, W, c->scratch));
    if (!c->hpin) {
        if (cudaMallocHost(&c->hpin, 1024 * sizeof(double)) != cudaSuccess) {
            c->err = "cudaMallocHost failed";
            return DC_ERR_OOM;
        }
        c->hpin_cap = 1024;
    }
    cudaError_t e = c->async_alloc ? ctx_sync(c, c->stream) : cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        c->err = std::string("device error during context creation: ") + cudaGetErrorString(e);
        return DC_ERR_CUDA;
    }
    return DC_OK;
}

dc_status prep_params_host(dc_ctx* c, std::vector<dc_params> q, ParamPrep& pp) {
    const int B = c->B;
    for (int i = 0; i < B; ++i) {
        std::string e = normalise_params(q[i]);
        if (!e.empty()) {
            c->err = "dc_set_params: " + e + (B > 1 ? " (instance " + std::to_string(i) + ")" : "");
            return DC_ERR_INVALID;
        }
        if (!same_batch_fields(q[i], q[0])) {
            c->err = "dc_set_params_batch: instance " + std::to_string(i) +
                     " differs from instance 0 in a field shared by the batch";
            return DC_ERR_INVALID;
        }
    }
    std::vector<HostFactor> hf(B);
    std::vector<HostFronts> fr(B);
    std::vector<HostPSolve> psi(B);
    std::vector<std::vector<double>> ccon(B);   // constant compliance per free node (not ROWSUM)
    std::vector<dc_status> st(B, DC_OK);
    std::vector<std::string> err(B);
    dc_parallel_for(B, [&](int i) {
        const HostMesh& h = c->ihm[i];
        std::vector<double> mass(h.m);
        for (int l = 0; l < h.m; ++l) mass[l] = q[i].density * h.abar[l];
        st[i] = dc_build_factor(h, q[i], mass, hf[i], err[i], q[i].factor_on_gpu == 1);
        if (st[i] == DC_OK && q[i].contact_compliance != DC_COMPLIANCE_ROWSUM) {
            // c_j per free node (internal order), reading of Eq. ly_et_al_govrningEq
            std::vector<double>& cv = ccon[i];
            cv.assign(h.m_free, 0.0);
            if (q[i].contact_compliance == DC_COMPLIANCE_DIAG_PINV) {
                std::vector<double> zd;
                dc_inverse_diagonal(hf[i], zd);
                for (int l = 0; l < h.m_free; ++l) cv[l] = q[i].h * zd[l];
            } else if (q[i].contact_compliance == DC_COMPLIANCE_DIAG_P) {
                for (int l = 0; l < h.m_free; ++l) cv[l] = q[i].h / hf[i].pdiag[l];
            } else {
                for (int l = 0; l < h.m_free; ++l) cv[l] = q[i].h / mass[l];
            }
        }
        if (st[i] == DC_OK) {
            std::string fe = dc_build_fronts(h, hf[i], fr[i]);
            if (!fe.empty()) {
                st[i] = DC_ERR_INVALID;
                err[i] = fe;
            } else if (q[i].global_solver == 1) {
                dc_build_psolve(hf[i], fr[i], psi[i], q[i].factor_on_gpu == 0);
            }
        }
        // only the explicit inverse rows, the size and the largest pivot are kept
        hf[i].rowidx = std::vector<int>();
        hf[i].val = std::vector<double>();
    });
    for (int i = 0; i < B; ++i)
        if (st[i]) {
            c->err = "dc_set_params: " + err[i] + (B > 1 ? " (instance " + std::to_string(i) + ")" : "");
            return st[i];
        }
    const HostMesh& hm = c->hm;
    const int MF = hm.m_free;
    std::vector<double> tau_i(B);
    for (int i = 0; i < B; ++i) tau_i[i] = 1e-7 * hf[i].max_diag;
    dc_merge_factors(hf, c->inst, pp.hfm);
    hf.clear();
    dc_merge_fronts(fr, c->inst, MF, pp.frm);
    fr.clear();
    if (q[0].global_solver == 1) dc_merge_psolve(psi, pp.ps);
    psi.clear();
    const HostFronts& frm = pp.frm;
    // per merged node / triangle material, per-instance tables
    pp.mass.assign(hm.m, 0.0);
    pp.wt.assign(hm.T, 0.0);
    pp.wb.assign(hm.m, 0.0);
    pp.node_mu.assign(hm.m, 0.0);
    pp.optr.assign(B + 1, 0);
    pp.okind.clear();
    pp.oprm.clear();
    pp.tau.assign(frm.S, 0.0f);
    pp.ccon.assign(q[0].contact_compliance != DC_COMPLIANCE_ROWSUM ? MF : 0, 0.0);
    for (int i = 0; i < B; ++i) {
        const InstInfo& in = c->inst[i];
        const HostMesh& h = c->ihm[i];
        if (!pp.ccon.empty())
            for (int l = 0; l < in.mf; ++l) pp.ccon[in.map(l, MF)] = ccon[i][l];
        for (int l = 0; l < in.m; ++l) {
            const int g = in.map(l, MF);
            pp.mass[g] = q[i].density * h.abar[l];
            pp.wb[g] = q[i].k_bend * h.abar[l];
            pp.node_mu[g] = q[i].mu;
        }
        for (int t = 0; t < in.T; ++t) pp.wt[in.to + t] = q[i].k_stretch * h.area[t];
        for (int o = 0; o < q[i].n_obstacles; ++o) {
            const dc_obstacle& ob = q[i].obstacles[o];
            pp.okind.push_back(ob.kind);
            if (ob.kind == DC_MESH) {
                const int id = (int)ob.p[0];
                if (id >= (int)c->mesh_t0.size()) {
                    c->err = "dc_set_params: obstacle mesh " + std::to_string(id) + " was not registered";
                    return DC_ERR_INVALID;
                }
                for (int k = 0; k < 8; ++k)
                    pp.oprm.push_back(k == 0 ? (double)c->mesh_t0[id] : (k == 1 ? (double)c->mesh_nt[id] : 0.0));
            } else {
                for (int k = 0; k < 8; ++k) pp.oprm.push_back(k < 7 ? ob.p[k] : 0.0);
            }
        }
        pp.optr[i + 1] = (int)pp.okind.size();
        const int S_i = (i + 1 < B ? c->inst[i + 1].so : frm.S) - in.so;
        for (int s = 0; s < S_i; ++s) pp.tau[in.so + s] = (float)tau_i[i];
    }
    pp.long_rows.clear();
    pp.short_rows.clear();
    for (int i = 0; i < MF; ++i)
        (pp.hfm.fptr[i + 1] - pp.hfm.fptr[i] > 1024 ? pp.long_rows : pp.short_rows).push_back(i);
    pp.front_flops = 0.0;
    for (int sn = 0; sn < frm.S; ++sn)
        for (int k = 0; k < frm.p[sn]; ++k) {
            double r = frm.f[sn] - k - 1;
            pp.front_flops += r + r * (r + 1.0);
        }
    pp.factor_nnz = pp.hfm.colptr.empty() ? 0 : pp.hfm.colptr.back();
    pp.q = std::move(q);
    return DC_OK;
}

dc_status upload_params(dc_ctx* c, ParamPrep& pp) {
    const HostMesh& hm = c->hm;
    const int MF = hm.m_free;
    HostFactor& hfm = pp.hfm;
    HostFronts& frm = pp.frm;
    free_pool(c, c->factor_allocs);
    c->graph_epoch++;
    c->have_params = false;
    auto& P = c->factor_allocs;
    double *d_mass, *d_wt, *d_wb, *d_fval, *d_kval, *d_mu, *d_oprm, *d_ccon = nullptr;
    d4* d_mesh = nullptr;
    int *d_fptr, *d_fidx, *d_kptr, *d_kidx, *d_long, *d_short, *d_optr, *d_okind;
    dc_status s;
    if ((s = upload(c, P, &d_mass, pp.mass)) || (s = upload(c, P, &d_wt, pp.wt)) || (s = upload(c, P, &d_wb, pp.wb)) ||
        (s = upload(c, P, &d_fptr, hfm.fptr)) || (s = upload(c, P, &d_fidx, hfm.fidx)) ||
        (s = upload(c, P, &d_fval, hfm.fval)) || (s = upload(c, P, &d_kptr, hfm.bptr)) ||
        (s = upload(c, P, &d_kidx, hfm.bidx)) || (s = upload(c, P, &d_kval, hfm.bval)) ||
        (s = upload(c, P, &d_long, pp.long_rows)) || (s = upload(c, P, &d_short, pp.short_rows)) ||
        (s = upload(c, P, &d_mu, pp.node_mu)) || (s = upload(c, P, &d_optr, pp.optr)) ||
        (s = upload(c, P, &d_okind, pp.okind)) || (s = upload(c, P, &d_oprm, pp.oprm)) ||
        (!pp.ccon.empty() && (s = upload(c, P, &d_ccon, pp.ccon))) ||
        (!c->mesh_rec.empty() && (s = upload(c, P, &d_mesh, c->mesh_rec))))
        return s;
    DevMesh& dm = c->dm;
    dm.n_long = (int)pp.long_rows.size();
    dm.n_short = (int)pp.short_rows.size();
    dm.long_rows = d_long;
    dm.short_rows = d_short;
    dm.mass = d_mass;
    dm.wt = d_wt;
    dm.wb = d_wb;
    dm.fptr = d_fptr;
    dm.fidx = d_fidx;
    dm.fval = d_fval;
    dm.kptr = d_kptr;
    dm.kidx = d_kidx;
    dm.kval = d_kval;
    DevParams& dp = c->dp;
    dp.h = pp.q[0].h;
    for (int k = 0; k < 3; ++k) dp.g[k] = pp.q[0].gravity[k];
    dp.delta = pp.q[0].contact_margin;
    dp.compliance = pp.q[0].contact_compliance;
    dp.mass_split = dp.compliance == DC_COMPLIANCE_MASS ? 1 : 0;
    dp.ccon = d_ccon;
    dp.mesh = d_mesh;
    dp.node_mu = d_mu;
    dp.optr = d_optr;
    dp.okind = d_okind;
    dp.oprm = d_oprm;
    // multifrontal structure for the adjoint preconditioner
    int dev = 0, smem_optin = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    // levels whose fronts do not fit one CTA's shared memory factorise with a
    // global scratch instead (the top fronts of large meshes)
    long gscr_floats = 0;
    size_t factor_bytes = 0;
    frontal_plan(frm, (size_t)smem_optin, &gscr_floats, &factor_bytes);
    if (frontal_solve_smem(frm.max_f) > (size_t)smem_optin) {
        c->err = "dc_set_params: the largest front (" + std::to_string(frm.max_f) +
                 " unknowns) exceeds the shared memory of one solve CTA";
        return DC_ERR_INVALID;
    }
    CK(frontal_configure(factor_bytes, frm.max_f));
    free_pool(c, c->front_allocs);
    auto& F = c->front_allocs;
    FrontDev fd{};
    fd.smem_limit = (size_t)smem_optin;
    fd.S = frm.S;
    fd.NP = (int)frm.pr_i.size();
    fd.max_f = frm.max_f;
    fd.pool_size = frm.pool_size;
    int *d_begin, *d_f, *d_p, *d_uptr, *d_unode, *d_cptr, *d_child, *d_cmap, *d_lvl, *d_pi, *d_pj, *d_pld, *d_pcp,
        *d_pcode;
    long long *d_off, *d_acc_off, *d_pdst, *d_binv_off, *d_linv_off;
    double* d_pcoef;
    float* d_tau;
    const size_t n3 = 3 * (size_t)std::max(MF, 1);
    std::vector<int> sn_inst(frm.S, 0);
    for (int i = 0; i < c->B; ++i) {
        const int end = i + 1 < c->B ? c->inst[i + 1].so : frm.S;
        for (int q = c->inst[i].so; q < end; ++q) sn_inst[q] = i;
    }
    int* d_sninst;
    if ((s = upload(c, F, &d_begin, frm.begin)) || (s = upload(c, F, &d_f, frm.f)) || (s = upload(c, F, &d_p, frm.p)) ||
        (s = upload(c, F, &d_off, frm.off)) || (s = upload(c, F, &d_acc_off, frm.acc_off)) ||
        (s = upload(c, F, &d_binv_off, frm.binv_off)) || (s = dalloc(c, F, &fd.binv, (size_t)frm.binv_size)) ||
        (s = upload(c, F, &d_linv_off, frm.linv_off)) || (s = dalloc(c, F, &fd.linv, (size_t)frm.linv_size)) ||
        (s = upload(c, F, &d_uptr, frm.uptr)) || (s = upload(c, F, &d_unode, frm.unode)) ||
        (s = upload(c, F, &d_cptr, frm.cptr)) || (s = upload(c, F, &d_child, frm.child)) ||
        (s = upload(c, F, &d_cmap, frm.cmap)) || (s = upload(c, F, &d_lvl, frm.lvl_sn)) ||
        (s = upload(c, F, &d_pi, frm.pr_i)) || (s = upload(c, F, &d_pj, frm.pr_j)) ||
        (s = upload(c, F, &d_pdst, frm.pr_dst)) || (s = upload(c, F, &d_pld, frm.pr_ld)) ||
        (s = upload(c, F, &d_pcp, frm.pr_cptr)) || (s = upload(c, F, &d_pcode, frm.pr_code)) ||
        (s = upload(c, F, &d_pcoef, frm.pr_coef)) || (s = upload(c, F, &d_tau, pp.tau)) ||
        (s = upload(c, F, &d_sninst, sn_inst)) ||
        (s = dalloc(c, F, &fd.pool, (size_t)frm.pool_size)) || (s = dalloc(c, F, &fd.acc, (size_t)frm.acc_size)) ||
        (s = dalloc(c, F, &fd.rvec, n3)) || (s = dalloc(c, F, &fd.zvec, n3)) || (s = dalloc(c, F, &fd.xvec, n3)))
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
    fd.tau = d_tau;
    fd.sn_inst = d_sninst;
    // tree-scheduled solves: the fronts in a topological order (children first);
    // DC_LEVEL_SOLVES=1 in the environment selects one launch per tree level
    // instead (same results)
    {
        std::vector<int> tq_ptr, tq_sn;
        dc_build_tree_items(frm, tq_ptr, tq_sn);
        // pull lists of the children's update vectors (float offsets of each node's x)
        std::vector<int> acc_base(frm.S), pull_off, pull_ptr, pull_idx;
        for (int q = 0; q < frm.S; ++q) acc_base[q] = (int)frm.acc_off[q];
        dc_build_pull_lists(frm, acc_base, 3, pull_off, pull_ptr, pull_idx);
        int *d_tq, *d_parent, *d_sched, *d_pull_off, *d_pull_ptr, *d_pull_idx;
        if ((s = upload(c, F, &d_tq, tq_sn)) || (s = upload(c, F, &d_parent, frm.parent)) ||
            (s = dalloc(c, F, &d_sched, 2 * ((size_t)frm.S + 1))) || (s = upload(c, F, &d_pull_off, pull_off)) ||
            (s = upload(c, F, &d_pull_ptr, pull_ptr)) || (s = upload(c, F, &d_pull_idx, pull_idx)))
            return s;
        fd.pull_off = d_pull_off;
        fd.pull_ptr = d_pull_ptr;
        fd.pull_idx = d_pull_idx;
        fd.tq = d_tq;
        fd.parent = d_parent;
        fd.sched = d_sched;
        fd.fault = c->counters + 3;
        fd.tree = std::getenv("DC_LEVEL_SOLVES") ? 0 : 1;
        CK(frontal_tree_grid(frm.max_f, &fd.tree_grid_f, &fd.tree_grid_b, &fd.tree_smem));
        c->tq_h = std::move(tq_sn);
        c->sn_inst_h = sn_inst;
    }
    c->fdv = fd;
    c->fds[0] = fd;
    c->fds[1] = fd;   // second slot: its own numeric storage, shared structure
    if ((s = dalloc(c, F, &c->fds[1].pool, (size_t)frm.pool_size)) ||
        (s = dalloc(c, F, &c->fds[1].binv, (size_t)frm.binv_size)) ||
        (s = dalloc(c, F, &c->fds[1].linv, (size_t)frm.linv_size)))
        return s;
    for (int k = 0; k < 2; ++k) {
        c->fds[k].gscr = nullptr;
        if (gscr_floats > 0 && (s = dalloc(c, F, &c->fds[k].gscr, (size_t)gscr_floats, false))) return s;
    }
    c->fdv = c->fds[0];
    // supernodal substitution of P (global_solver 1) on the same partition
    dm.solver = pp.q[0].global_solver;
    if (dm.solver == 1) {
        long long *d_poff, *d_xoff, *d_toff;
        int* d_aoff;
        double *d_panel, *d_xinv, *d_pant, *d_xinvt;
        d4 *d_acc, *d_xint;
        if ((s = upload(c, F, &d_poff, pp.ps.poff)) || (s = upload(c, F, &d_xoff, pp.ps.xoff)) ||
            (s = upload(c, F, &d_toff, pp.ps.toff)) || (s = upload(c, F, &d_aoff, pp.ps.aoff)) ||
            (pp.ps.panel.empty()   // factor_on_gpu: the GPU factorisation fills them below
                 ? ((s = dalloc(c, F, &d_panel, (size_t)std::max<long long>(pp.ps.n_panel, 1), false)) ||
                    (s = dalloc(c, F, &d_xinv, (size_t)std::max<long long>(pp.ps.n_xinv, 1), false)) ||
                    (s = dalloc(c, F, &d_pant, (size_t)std::max<long long>(pp.ps.n_pant, 1), false)) ||
                    (s = dalloc(c, F, &d_xinvt, (size_t)std::max<long long>(pp.ps.n_xinv, 1), false)))
                 : ((s = upload(c, F, &d_panel, pp.ps.panel)) || (s = upload(c, F, &d_xinv, pp.ps.xinv)) ||
                    (s = upload(c, F, &d_pant, pp.ps.pant)) || (s = upload(c, F, &d_xinvt, pp.ps.xinvt)))) ||
            (s = dalloc(c, F, &d_acc, (size_t)std::max<long long>(pp.ps.acc_nodes, 1))) ||
            (s = dalloc(c, F, &d_xint, (size_t)std::max(MF, 1))))
            return s;
        // per level: the large fronts (CTA path) first, then the small ones (warp path)
        std::vector<int> psn(frm.S);
        const int nl = (int)frm.lvl_ptr.size() - 1;
        c->ps_lvl_ptr.assign(nl + 1, 0);
        c->ps_nbig.assign(nl, 0);
        c->ps_nsmall.assign(nl, 0);
        c->ps_maxbig.assign(nl, 0);
        int pos = 0;
        for (int l = 0; l < nl; ++l) {
            c->ps_lvl_ptr[l] = pos;
            for (int q = frm.lvl_ptr[l]; q < frm.lvl_ptr[l + 1]; ++q) {
                const int sn = frm.lvl_sn[q], fsn = frm.f[sn] / 3;
                if (fsn > DC_PS_SMALL) {
                    psn[pos++] = sn;
                    c->ps_maxbig[l] = std::max(c->ps_maxbig[l], fsn);
                }
            }
            c->ps_nbig[l] = pos - c->ps_lvl_ptr[l];
            for (int q = frm.lvl_ptr[l]; q < frm.lvl_ptr[l + 1]; ++q) {
                const int sn = frm.lvl_sn[q];
                if (frm.f[sn] / 3 <= DC_PS_SMALL) psn[pos++] = sn;
            }
            c->ps_nsmall[l] = pos - c->ps_lvl_ptr[l] - c->ps_nbig[l];
        }
        c->ps_lvl_ptr[nl] = pos;
        int* d_psn;
        if ((s = upload(c, F, &d_psn, psn))) return s;
        std::vector<int> tq_ptr, tq_sn;
        dc_build_tree_items(frm, tq_ptr, tq_sn);
        std::vector<int> pull_off, pull_ptr, pull_idx;
        dc_build_pull_lists(frm, pp.ps.aoff, 1, pull_off, pull_ptr, pull_idx);
        int *d_tq_ptr, *d_tq_sn, *d_sched, *d_pull_off, *d_pull_ptr, *d_pull_idx;
        if ((s = upload(c, F, &d_tq_ptr, tq_ptr)) || (s = upload(c, F, &d_tq_sn, tq_sn)) ||
            (s = dalloc(c, F, &d_sched, 2 * ((size_t)frm.S + 1))) || (s = upload(c, F, &d_pull_off, pull_off)) ||
            (s = upload(c, F, &d_pull_ptr, pull_ptr)) || (s = upload(c, F, &d_pull_idx, pull_idx)))
            return s;
        PSolveDev& ps = dm.ps;
        ps.S = frm.S;
        ps.n_items = (int)tq_ptr.size() - 1;
        ps.parent = fd.parent;
        ps.tq_ptr = d_tq_ptr;
        ps.tq_sn = d_tq_sn;
        ps.sched = d_sched;
        ps.pull_off = d_pull_off;
        ps.pull_ptr = d_pull_ptr;
        ps.pull_idx = d_pull_idx;
        ps.fault = c->counters + 3;
        ps.tree = fd.tree;
        // both sweeps of a global step in one launch (DC_SEPARATE_SWEEPS=1 in the
        // environment: two launches, for comparison; the same results)
        ps.fused = std::getenv("DC_SEPARATE_SWEEPS") ? 0 : 1;
        ps.sn = d_psn;
        ps.begin = d_begin;
        ps.f = d_f;
        ps.p = d_p;
        ps.uptr = d_uptr;
        ps.unode = d_unode;
        ps.cptr = d_cptr;
        ps.child = d_child;
        ps.cmap = d_cmap;
        ps.poff = d_poff;
        ps.xoff = d_xoff;
        ps.toff = d_toff;
        ps.aoff = d_aoff;
        ps.panel = d_panel;
        ps.xinv = d_xinv;
        ps.pant = d_pant;
        ps.xinvt = d_xinvt;
        ps.acc = d_acc;
        ps.xint = d_xint;
    }
    c->psolve_flops = 0.0;
    if (dm.solver == 1)
        for (int q = 0; q < frm.S; ++q) {
            const double ns = frm.p[q] / 3, nu = (frm.f[q] - frm.p[q]) / 3;
            c->psolve_flops += 6.0 * (ns * (ns + 1.0) / 2.0 + ns * nu);   // 3 columns, one FMA = 2 flops
        }
    c->nlev = (int)frm.lvl_ptr.size() - 1;
    c->lvl_maxf.assign(std::max(c->nlev, 0), 0);
    c->lvl_maxp.assign(std::max(c->nlev, 0), 0);
    for (int l = 0; l < c->nlev; ++l)
        for (int q = frm.lvl_ptr[l]; q < frm.lvl_ptr[l + 1]; ++q)
            c->lvl_maxf[l] = std::max(c->lvl_maxf[l], frm.f[frm.lvl_sn[q]]);
    for (int l = 0; l < c->nlev; ++l)
        for (int q = frm.lvl_ptr[l]; q < frm.lvl_ptr[l + 1]; ++q)
            c->lvl_maxp[l] = std::max(c->lvl_maxp[l], frm.p[frm.lvl_sn[q]]);
    c->front_flops = pp.front_flops;
    c->factor_nnz = pp.factor_nnz;
    c->fwd_nnz = (long long)hfm.fval.size();
    c->bwd_nnz = (long long)hfm.bval.size();
    c->hf = HostFactor();
    c->hf.max_diag = hfm.max_diag;
    c->fr = std::move(frm);
    c->lvl_maxfs.assign(c->lvl_maxf.size(), 0);
    for (size_t l = 0; l < c->lvl_maxf.size(); ++l) c->lvl_maxfs[l] = c->lvl_maxf[l] / 3;
    if (dm.solver == 1) {
        dm.ps.nlev = c->nlev;
        dm.ps.lvl_ptr_h = c->ps_lvl_ptr.data();
        dm.ps.nbig_h = c->ps_nbig.data();
        dm.ps.nsmall_h = c->ps_nsmall.data();
        dm.ps.maxbig_h = c->ps_maxbig.data();
        int mx = 0;
        for (int v : c->ps_maxbig) mx = std::max(mx, v);
        CK(psolve_configure(mx));
        CK(psolve_tree_grid(mx, &dm.ps.tree_grid_f, &dm.ps.tree_grid_b, &dm.ps.tree_smem));
    }
    {
        // per level, where each instance's fronts start in lvl_sn (an instance's
        // fronts are contiguous and ascending inside a level)
        const int B = c->B, nl = c->nlev;
        c->lvl_inst_ptr.assign((size_t)nl * (B + 1), 0);
        for (int l = 0; l < nl; ++l) {
            int* P = c->lvl_inst_ptr.data() + (size_t)l * (B + 1);
            int q = c->fr.lvl_ptr[l];
            for (int i = 0; i <= B; ++i) {
                while (q < c->fr.lvl_ptr[l + 1] && sn_inst[c->fr.lvl_sn[q]] < i) ++q;
                P[i] = q;
            }
            P[B] = c->fr.lvl_ptr[l + 1];
        }
    }
    if (pp.q[0].factor_on_gpu == 1) RET(gpu_factor_P(c, c->fr, pp.q[0].h));
    c->prm = pp.q[0];
    c->iprm = pp.q;
    c->have_params = true;
    c->ck_n_steps = -1;
    if (c->async_alloc) CK(ctx_sync(c, c->stream));
    return DC_OK;
}

size_t estimate_device_bytes(const dc_ctx* c, const MeshPrep& mp, const ParamPrep& pp, int n_steps) {
    const HostMesh& hm = c->hm;
    const size_t m = hm.m, T = hm.T, MF = hm.m_free, B = c->B;
    const size_t d4b = sizeof(d4);
    const dc_params& q = pp.q[0];
    const size_t k = std::max(1, q.checkpoint_every);
    const size_t mr = std::max(1, std::min(256, q.adj_restart));
    size_t b = 0, n = 0;   // bytes and allocation count (each rounded up below)
    auto add = [&](size_t bytes) {
        b += std::max<size_t>(bytes, 32);
        ++n;
    };
    // mesh
    add(vbytes(mp.tri4)); add(vbytes(mp.G4)); add(vbytes(hm.area)); add(vbytes(hm.bptr)); add(vbytes(hm.bidx));
    add(vbytes(hm.bval)); add(vbytes(hm.abar)); add(vbytes(hm.sb)); add(vbytes(mp.qr)); add(vbytes(mp.iptr));
    add(vbytes(mp.iidx)); add(vbytes(mp.tbptr)); add(vbytes(mp.tbidx)); add(vbytes(mp.tbval));
    add(vbytes(hm.int2ext)); add(vbytes(mp.node_inst)); add(vbytes(mp.cptr)); add(vbytes(mp.pcptr));
    add(vbytes(mp.chunks)); add(vbytes(mp.pchunks));
    // forward work
    for (int i = 0; i < 9; ++i) add(m * d4b);
    add(T * d4b); add(T * d4b); add(m * 8); add(m * 24); add(m * 24); add(64);
    add(MF * 4); add(MF * 4); add(MF * d4b); add(MF * d4b);
    // factor and tables
    const HostFactor& f = pp.hfm;
    add(vbytes(pp.mass)); add(vbytes(pp.wt)); add(vbytes(pp.wb)); add(vbytes(f.fptr)); add(vbytes(f.fidx));
    add(vbytes(f.fval)); add(vbytes(f.bptr)); add(vbytes(f.bidx)); add(vbytes(f.bval)); add(vbytes(pp.long_rows));
    add(vbytes(pp.short_rows)); add(vbytes(pp.node_mu)); add(vbytes(pp.optr)); add(vbytes(pp.okind));
    add(vbytes(pp.oprm));
    if (!pp.ccon.empty()) add(vbytes(pp.ccon));
    // fronts (numeric storage twice: two slots)
    const HostFronts& r = pp.frm;
    add(vbytes(r.begin)); add(vbytes(r.f)); add(vbytes(r.p)); add(vbytes(r.off)); add(vbytes(r.acc_off));
    add(vbytes(r.binv_off)); add(vbytes(r.linv_off)); add(vbytes(r.uptr)); add(vbytes(r.unode)); add(vbytes(r.cptr));
    add(vbytes(r.child)); add(vbytes(r.cmap)); add(vbytes(r.lvl_sn)); add(vbytes(r.pr_i)); add(vbytes(r.pr_j));
    add(vbytes(r.pr_dst)); add(vbytes(r.pr_ld)); add(vbytes(r.pr_cptr)); add(vbytes(r.pr_code));
    add(vbytes(r.pr_coef)); add(vbytes(pp.tau)); add(vbytes(pp.tau));
    long gscr_floats = 0;
    size_t factor_bytes = 0;
    int dev = 0, optin = 227 * 1024;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        optin = 227 * 1024;   // host-only estimate without a device: the GB300 limit
    }
    frontal_plan(r, (size_t)optin, &gscr_floats, &factor_bytes);
    for (int s = 0; s < 2; ++s) {
        add(4 * (size_t)r.pool_size);
        add(4 * (size_t)r.binv_size);
        add(4 * (size_t)r.linv_size);
        if (gscr_floats > 0) add(4 * (size_t)gscr_floats);
    }
    add(4 * (size_t)r.acc_size); add(12 * MF); add(12 * MF); add(12 * MF);
    add(4 * (size_t)r.S); add(4 * (size_t)r.S); add(8 * ((size_t)r.S + 1));   // tree order, parents, tickets/flags
    {
        size_t nodes = 0;   // pull lists of the children's update vectors
        for (int q = 0; q < r.S; ++q) nodes += r.f[q] / 3 + 1;
        add(4 * (size_t)r.S); add(4 * nodes); add(4 * (size_t)r.acc_size / 3 + 4);
    }
    if (q.global_solver == 1) {
        add(vbytes(pp.ps.poff)); add(vbytes(pp.ps.xoff)); add(vbytes(pp.ps.toff)); add(vbytes(pp.ps.aoff));
        add(8 * (size_t)pp.ps.n_panel); add(8 * (size_t)pp.ps.n_xinv); add(8 * (size_t)pp.ps.n_pant);
        add(8 * (size_t)pp.ps.n_xinv);
        add(vbytes(pp.ps.aoff));
        if (q.factor_on_gpu == 1) {   // temporary node-level fronts, their offsets and pair destinations
            size_t ff = 0;
            for (int s = 0; s < r.S; ++s) ff += (size_t)(r.f[s] / 3) * (r.f[s] / 3);
            add(8 * ff); add(8 * ((size_t)r.S + 1)); add(8 * r.pr_i.size());
        }
        add((size_t)pp.ps.acc_nodes * d4b); add(MF * d4b);
        // tree schedule: items (at most one per front), two ticket/flag arrays
        add(4 * ((size_t)r.S + 1)); add(4 * (size_t)r.S); add(8 * ((size_t)r.S + 1));
        // pull lists of the child gather
        size_t nodes = 0;
        for (int q = 0; q < r.S; ++q) nodes += r.f[q] / 3 + 1;
        add(4 * (size_t)r.S); add(4 * nodes); add(4 * (size_t)pp.ps.acc_nodes);
    }
    // checkpoints, segment recomputation, adjoint
    add(((size_t)n_steps / k + 1) * 2 * m * d4b);
    if (k == 1)
        for (int i = 0; i < n_steps; ++i) { add(MF * 4); add(MF * 4); add(MF * d4b); add(MF * d4b); }
    add((k + 1) * m * d4b); add((k + 1) * m * d4b);
    for (size_t i = 0; i < k; ++i) { add(MF * 4); add(MF * 4); add(MF * d4b); add(MF * d4b); }
    add(T * d4b); add(T * d4b); add(m * d4b);
    for (int s = 0; s < 2; ++s) {
        add(T * d4b); add(T * d4b); add(T * d4b); add(4 * T * d4b); add(m * d4b); add(3 * MF * d4b); add(MF * d4b);
        add(MF * 4);
    }
    for (int i = 0; i < 15; ++i) add(m * d4b);
    add((mr + 1) * 4 * m * 8); add(mr * 4 * m * 8); add((mr + 1) * B * 8); add((mr + 1) * B * 8);
    add(B * 8); add(B * 8); add((mr + 1) * mp.chunks.size() * 8); add(4 * B * 8); add(mp.pchunks.size() * 8);
    // allocation granularity of the device pools
    return b + n * 512;
}
