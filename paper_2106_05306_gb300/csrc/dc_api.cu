// C ABI of libdc: context creation (one cloth or a batch of cloths packed into
// one disconnected problem), parameters and factorisation, the forward step /
// rollout and the checkpointed backward pass.  The time stepping and the
// adjoint Krylov solve are in dc_driver.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "dc_ctx.h"
#include "dc_obstacle.cuh"

namespace {

std::string g_create_err;

dc_status create_common(dc_ctx* c) {
    MeshPrep mp;
    prep_mesh_host(c, mp);
    return upload_mesh(c, mp);
}

dc_status finish_create(dc_ctx* c, dc_ctx** out, void* stream) {
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        g_create_err = "no usable CUDA device";
        delete c;
        return DC_ERR_CUDA;
    }
    c->kt.stream = c->stream;
    dc_status s = create_common(c);
    if (s) {
        g_create_err = c->err;
        free_pool(c, c->work_allocs);
        free_pool(c, c->mesh_allocs);
        if (c->hpin) cudaFreeHost(c->hpin);
        delete c;
        return s;
    }
    *out = c;
    return DC_OK;
}

// Per-instance parameters: host factorisations (threads), then the upload.
dc_status apply_params(dc_ctx* c, std::vector<dc_params> q) {
    ParamPrep pp;
    RET(prep_params_host(c, std::move(q), pp));
    CK(ctx_sync(c, c->stream));   // earlier work may still read the old factor
    return upload_params(c, pp);
}

}  // namespace

// Device-side error words, read after the stream's work so far: the sticky
// fault word of the bounded waits (counters[3], DC_ERR_TIMEOUT: every result
// computed since is invalid) and the non-finite forward state flag
// (counters[4], DC_ERR_NONFINITE, cleared once reported).
dc_status check_device_flags(dc_ctx* c) {
    if (!c->counters) return DC_OK;
    unsigned long long w[2] = {0, 0};
    CK(cudaMemcpyAsync(w, c->counters + 3, sizeof(w), cudaMemcpyDeviceToHost, c->stream));
    CK(ctx_sync(c, c->stream));
    if (w[0]) {
        c->err = "a bounded device wait (a dependency flag or a tensor-core completion) gave up; results since then are invalid";
        return DC_ERR_TIMEOUT;
    }
    if (w[1]) {
        CK(cudaMemsetAsync(c->counters + 4, 0, sizeof(unsigned long long), c->stream));
        CK(ctx_sync(c, c->stream));
        c->err = "a forward step produced a non-finite position or velocity";
        return DC_ERR_NONFINITE;
    }
    return DC_OK;
}

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
    p->contact_compliance = DC_COMPLIANCE_ROWSUM;
    p->adj_fallback = 1;
}

dc_status dc_set_instance_steps(dc_ctx* c, const int32_t* steps) {
    if (!c) return DC_ERR_INVALID;
    if (!steps) {
        c->inst_steps.clear();
        c->d_inst_steps = nullptr;   // the device copy stays in work_allocs until dc_destroy
        c->graph_epoch++;
        return DC_OK;
    }
    for (int i = 0; i < c->B; ++i)
        if (steps[i] < 0) {
            c->err = "dc_set_instance_steps: negative step count";
            return DC_ERR_INVALID;
        }
    c->inst_steps.assign(steps, steps + c->B);
    // B step counts, then the first step of the segment a recomputation replays
    if (!c->d_inst_steps_buf) RET(dalloc(c, c->work_allocs, &c->d_inst_steps_buf, (size_t)c->B + 1));
    CK(cudaMemcpyAsync(c->d_inst_steps_buf, c->inst_steps.data(), sizeof(int) * c->B, cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemsetAsync(c->d_inst_steps_buf + c->B, 0, sizeof(int), c->stream));
    CK(ctx_sync(c, c->stream));
    c->d_inst_steps = c->d_inst_steps_buf;
    c->graph_epoch++;
    return DC_OK;
}

dc_status dc_add_obstacle_mesh(dc_ctx* c, int32_t nv, const double* verts, int32_t nt, const int32_t* tris,
                               int32_t* mesh_id) {
    if (!c) return DC_ERR_INVALID;
    if (nv < 3 || nt < 4 || !verts || !tris || !mesh_id) {
        c->err = "dc_add_obstacle_mesh: a closed mesh needs at least 4 triangles and 3 vertices";
        return DC_ERR_INVALID;
    }
    for (long k = 0; k < 3L * nv; ++k)
        if (!std::isfinite(verts[k])) {
            c->err = "dc_add_obstacle_mesh: non-finite vertex";
            return DC_ERR_INVALID;
        }
    // closed and consistently oriented: every directed edge once, with its reverse once
    std::vector<std::pair<long long, int>> dir;
    dir.reserve(3 * (size_t)nt);
    for (int t = 0; t < nt; ++t)
        for (int k = 0; k < 3; ++k) {
            const int i = tris[3 * t + k], j = tris[3 * t + (k + 1) % 3];
            if (i < 0 || i >= nv || j < 0 || j >= nv || i == j) {
                c->err = "dc_add_obstacle_mesh: bad vertex index in triangle " + std::to_string(t);
                return DC_ERR_INVALID;
            }
            dir.push_back({(long long)i * nv + j, t});
        }
    std::sort(dir.begin(), dir.end());
    for (size_t q = 0; q < dir.size(); ++q) {
        const long long e = dir[q].first, rev = (e % nv) * nv + e / nv;
        const bool dup = (q > 0 && dir[q - 1].first == e) || (q + 1 < dir.size() && dir[q + 1].first == e);
        const auto it = std::lower_bound(dir.begin(), dir.end(), std::make_pair(rev, -1));
        if (dup || it == dir.end() || it->first != rev) {
            c->err = "dc_add_obstacle_mesh: the mesh is not closed and consistently oriented";
            return DC_ERR_INVALID;
        }
    }
    auto V = [&](int i, int k) { return verts[3 * (long)i + k]; };
    std::vector<double> fn(3 * (size_t)nt), vn(3 * (size_t)nv, 0.0);
    for (int t = 0; t < nt; ++t) {
        const int a = tris[3 * t], b = tris[3 * t + 1], cc = tris[3 * t + 2];
        double u[3], w[3];
        for (int k = 0; k < 3; ++k) { u[k] = V(b, k) - V(a, k); w[k] = V(cc, k) - V(a, k); }
        double n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
        const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(nn > 0.0)) {
            c->err = "dc_add_obstacle_mesh: degenerate triangle " + std::to_string(t);
            return DC_ERR_INVALID;
        }
        for (int k = 0; k < 3; ++k) fn[3 * t + k] = n[k] / nn;
        // angle-weighted vertex pseudo-normals
        const int idx[3] = {a, b, cc};
        for (int q = 0; q < 3; ++q) {
            const int i = idx[q], j = idx[(q + 1) % 3], l = idx[(q + 2) % 3];
            double p1[3], p2[3];
            for (int k = 0; k < 3; ++k) { p1[k] = V(j, k) - V(i, k); p2[k] = V(l, k) - V(i, k); }
            const double cs = (p1[0] * p2[0] + p1[1] * p2[1] + p1[2] * p2[2]) /
                              (std::sqrt(p1[0] * p1[0] + p1[1] * p1[1] + p1[2] * p1[2]) *
                               std::sqrt(p2[0] * p2[0] + p2[1] * p2[1] + p2[2] * p2[2]));
            const double ang = std::acos(std::max(-1.0, std::min(1.0, cs)));
            for (int k = 0; k < 3; ++k) vn[3 * (size_t)i + k] += ang * fn[3 * t + k];
        }
    }
    // the triangle on the other side of each directed edge
    auto other = [&](int i, int j) {
        const auto it = std::lower_bound(dir.begin(), dir.end(), std::make_pair((long long)j * nv + i, -1));
        return it->second;
    };
    const int t0 = (int)(c->mesh_rec.size() / DC_MESH_REC);
    for (int t = 0; t < nt; ++t) {
        const int idx[3] = {tris[3 * t], tris[3 * t + 1], tris[3 * t + 2]};
        for (int q = 0; q < 3; ++q) c->mesh_rec.push_back(d4{V(idx[q], 0), V(idx[q], 1), V(idx[q], 2), 0.0});
        c->mesh_rec.push_back(d4{fn[3 * t], fn[3 * t + 1], fn[3 * t + 2], 0.0});
        for (int q = 0; q < 3; ++q) {   // edges AB, BC, CA
            const int u = other(idx[q], idx[(q + 1) % 3]);
            c->mesh_rec.push_back(d4{fn[3 * t] + fn[3 * u], fn[3 * t + 1] + fn[3 * u + 1],
                                     fn[3 * t + 2] + fn[3 * u + 2], 0.0});
        }
        for (int q = 0; q < 3; ++q)
            c->mesh_rec.push_back(d4{vn[3 * (size_t)idx[q]], vn[3 * (size_t)idx[q] + 1], vn[3 * (size_t)idx[q] + 2], 0.0});
    }
    c->mesh_t0.push_back(t0);
    c->mesh_nt.push_back(nt);
    *mesh_id = (int32_t)c->mesh_t0.size() - 1;
    return DC_OK;
}

dc_status dc_set_layout(dc_ctx* c, int32_t layout) {
    if (!c) return DC_ERR_INVALID;
    if (layout != DC_LAYOUT_NODE_MAJOR && layout != DC_LAYOUT_COMPONENT_MAJOR) {
        c->err = "dc_set_layout: unknown layout";
        return DC_ERR_INVALID;
    }
    c->layout = layout;
    return DC_OK;
}

dc_status dc_batch_hbm_bytes(int32_t n, const dc_instance* in, const dc_params* params, int32_t n_steps,
                             int64_t* bytes) {
    if (n < 1 || !in || !params || !bytes || n_steps < 0) {
        g_create_err = "dc_batch_hbm_bytes: null argument, no instances or negative step count";
        return DC_ERR_INVALID;
    }
    for (int i = 0; i < n; ++i)
        if (!in[i].rest_pos || !in[i].tris || in[i].n_pins < 0 || (in[i].n_pins > 0 && !in[i].pins) ||
            in[i].n_nodes < 0) {
            g_create_err = "dc_batch_hbm_bytes: null argument (instance " + std::to_string(i) + ")";
            return DC_ERR_INVALID;
        }
    // the host half of dc_create_batch + dc_set_params_batch, no device work
    dc_ctx* c = new dc_ctx();
    c->ihm.resize(n);
    std::vector<std::string> err(n);
    dc_parallel_for(n, [&](int i) {
        err[i] = dc_build_mesh(c->ihm[i], in[i].n_nodes, in[i].rest_pos, in[i].n_tris, in[i].tris, in[i].n_pins,
                               in[i].pins);
    });
    for (int i = 0; i < n; ++i)
        if (!err[i].empty()) {
            g_create_err = "dc_batch_hbm_bytes: instance " + std::to_string(i) + ": " + err[i];
            delete c;
            return DC_ERR_INVALID;
        }
    MeshPrep mp;
    prep_mesh_host(c, mp);
    ParamPrep pp;
    dc_status s = prep_params_host(c, std::vector<dc_params>(params, params + n), pp);
    if (s) {
        g_create_err = "dc_batch_hbm_bytes: " + c->err;
        delete c;
        return s;
    }
    *bytes = (int64_t)estimate_device_bytes(c, mp, pp, n_steps);
    delete c;
    return DC_OK;
}

dc_status dc_create_mesh(dc_ctx** out, int32_t n_nodes, const double* rest_pos, int32_t n_tris,
                         const int32_t* tris, int32_t n_pins, const int32_t* pins, void* stream) {
    if (!out || !rest_pos || !tris || n_pins < 0 || (n_pins > 0 && !pins)) {
        g_create_err = "dc_create_mesh: null argument";
        return DC_ERR_INVALID;
    }
    *out = nullptr;
    dc_ctx* c = new dc_ctx();
    c->ihm.resize(1);
    std::string e = dc_build_mesh(c->ihm[0], n_nodes, rest_pos, n_tris, tris, n_pins, pins);
    if (!e.empty()) {
        g_create_err = "dc_create_mesh: " + e;
        delete c;
        return DC_ERR_INVALID;
    }
    return finish_create(c, out, stream);
}

dc_status dc_create_batch(dc_ctx** out, int32_t n, const dc_instance* in, void* stream) {
    if (!out || n < 1 || !in) {
        g_create_err = "dc_create_batch: null argument or no instances";
        return DC_ERR_INVALID;
    }
    *out = nullptr;
    long long total = 0;
    for (int i = 0; i < n; ++i) {
        if (!in[i].rest_pos || !in[i].tris || in[i].n_pins < 0 || (in[i].n_pins > 0 && !in[i].pins) ||
            in[i].n_nodes < 0) {
            g_create_err = "dc_create_batch: null argument (instance " + std::to_string(i) + ")";
            return DC_ERR_INVALID;
        }
        total += in[i].n_nodes;
    }
    if (total > (1LL << 28)) {
        g_create_err = "dc_create_batch: more than 2^28 nodes in one batch";
        return DC_ERR_INVALID;
    }
    dc_ctx* c = new dc_ctx();
    c->ihm.resize(n);
    std::vector<std::string> err(n);
    dc_parallel_for(n, [&](int i) {
        err[i] = dc_build_mesh(c->ihm[i], in[i].n_nodes, in[i].rest_pos, in[i].n_tris, in[i].tris, in[i].n_pins,
                               in[i].pins);
    });
    for (int i = 0; i < n; ++i)
        if (!err[i].empty()) {
            g_create_err = "dc_create_batch: instance " + std::to_string(i) + ": " + err[i];
            delete c;
            return DC_ERR_INVALID;
        }
    return finish_create(c, out, stream);
}

dc_status dc_get_layout(dc_ctx* c, int32_t* n_instances, int64_t* node_offsets) {
    if (!c || !n_instances) return DC_ERR_INVALID;
    *n_instances = c->B;
    if (node_offsets) {
        for (int i = 0; i < c->B; ++i) node_offsets[i] = c->inst[i].ext_off;
        node_offsets[c->B] = c->hm.m;
    }
    return DC_OK;
}

dc_status dc_set_params(dc_ctx* c, const dc_params* p) {
    if (!c || !p) return DC_ERR_INVALID;
    return apply_params(c, std::vector<dc_params>(c->B, *p));
}

dc_status dc_set_params_batch(dc_ctx* c, int32_t n, const dc_params* p) {
    if (!c || !p) return DC_ERR_INVALID;
    if (n != c->B) {
        c->err = "dc_set_params_batch: " + std::to_string(n) + " parameter sets for " + std::to_string(c->B) +
                 " instances";
        return DC_ERR_INVALID;
    }
    return apply_params(c, std::vector<dc_params>(p, p + n));
}

dc_status dc_set_graphs(dc_ctx* c, int32_t enable) {
    if (!c || (enable != 0 && enable != 1)) return DC_ERR_INVALID;
    c->use_graphs = enable == 1;
    return DC_OK;
}

dc_status dc_autotune(dc_ctx* c) {
    if (!c) return DC_ERR_INVALID;
    if (!c->have_params) {
        c->err = "dc_autotune: call dc_set_params first";
        return DC_ERR_STATE;
    }
    return autotune(c);
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
    c->steps++;
    RET(store_vec(c, c->xb, x_np1, host_io));
    RET(store_vec(c, c->vb, v_np1, host_io));
    CK(cudaGetLastError());
    if (host_io) RET(check_device_flags(c));
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
    if (k == 1) RET(ensure_records(c, n_steps));
    bool host_io = false;
    d4* X = c->ck;              // checkpoint 0 holds (x0, v0)
    d4* Vv = c->ck + m;
    RET(load_vec(c, x0, X, host_io));
    RET(load_vec(c, v0, Vv, host_io));
    launch_zero_pins(Vv, c->hm.m_free, m, c->stream);
    if (traj_x) {
        // with a trajectory output every step is stored: no graph
        bool h2 = false;
        RET(store_vec(c, X, traj_x, h2));
        host_io |= h2;
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
            run_step(c, cx, cv, nx, nv, k == 1 ? c->rec_all[s] : c->scratch, true, s);
            RET(store_vec(c, nx, traj_x + (size_t)(s + 1) * 3 * m, h2));
            host_io |= h2;
            cx = nx;
            cv = nv;
        }
        RET(store_vec(c, cx, x_final, host_io));
        RET(store_vec(c, cv, v_final, host_io));
    } else {
        RET(rollout_steps(c, n_steps, k));
        RET(store_vec(c, c->xa, x_final, host_io));
        RET(store_vec(c, c->va, v_final, host_io));
    }
    c->steps += n_steps;
    CK(cudaGetLastError());
    c->ck_n_steps = n_steps;
    c->ck_every = k;
    if (host_io) RET(check_device_flags(c));
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
    const int N = c->ck_n_steps, k = c->ck_every, m = c->hm.m, B = c->B;
    cudaStream_t s = c->stream;
    // k == 1: every step's state and record were kept by the rollout
    const bool direct = k == 1;
    if (!direct) RET(ensure_segment(c, k));
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
    Pool tmp;
    if (traj && !is_device_ptr(traj)) {
        RET(dalloc(c, tmp, &traj_dev, (size_t)(N + 1) * 3 * m, false));
        CK(cudaMemcpyAsync(traj_dev, traj, sizeof(double) * (N + 1) * 3 * m, cudaMemcpyHostToDevice, s));
        traj = traj_dev;
        host_io = true;
    }
    CK(cudaMemsetAsync(c->dparam_acc, 0, 4 * sizeof(double) * B, s));
    bool noncv = false;
    dc_status st = DC_OK;
    // direct: one segment over the whole rollout, so that the preparation of every
    // step overlaps the GMRES of the step after it
    const int n_seg = direct ? (N > 0 ? 1 : 0) : (N + k - 1) / k;
    for (int seg = n_seg - 1; seg >= 0 && st == DC_OK; --seg) {
        const int s0 = direct ? 0 : seg * k, s1 = direct ? N : std::min(N, s0 + k);
        if (!direct) {
            st = recompute_segment(c, seg, s0, s1);
            if (st) break;
        }
        // state x_t / v_t and the record of step t (t -> t+1), t in [s0, s1]
        auto X = [&](int t) -> const d4* {
            return direct ? c->ck + (size_t)t * 2 * m : c->segX + (size_t)(t - s0) * m;
        };
        auto V = [&](int t) -> const d4* {
            return direct ? c->ck + (size_t)t * 2 * m + m : c->segV + (size_t)(t - s0) * m;
        };
        auto R = [&](int t) -> const StepRec& { return direct ? c->rec_all[t] : c->seg_rec[t - s0]; };
        // step t's data is prepared on stream2 while the GMRES of step t+1 runs on
        // the main stream; slot t % 2 alternates between consecutive steps
        CK(cudaEventRecord(c->ev_seg, s));
        CK(cudaStreamWaitEvent(c->stream2, c->ev_seg, 0));
        {
            const int t = s1 - 1, k2 = t % 2;
            CK(cudaStreamWaitEvent(c->stream2, c->ev_free[k2], 0));
            prepare_step(c, R(t), X(t + 1), V(t + 1), k2, c->stream2);
            CK(cudaEventRecord(c->ev_fact[k2], c->stream2));
        }
        for (int t = s1 - 1; t >= s0; --t) {
            const int k2 = t % 2;
            if (t > s0) {
                const int kn = (t - 1) % 2;
                CK(cudaStreamWaitEvent(c->stream2, c->ev_free[kn], 0));
                prepare_step(c, R(t - 1), X(t), V(t), kn, c->stream2);
                CK(cudaEventRecord(c->ev_fact[kn], c->stream2));
            }
            CK(cudaStreamWaitEvent(s, c->ev_fact[k2], 0));
            if (traj) adj_add_ext(c->gx, traj + (size_t)(t + 1) * 3 * m, c->d_int2ext, m, c->layout, s);
            st = adjoint_step(c, X(t), X(t + 1), V(t + 1), k2, noncv, t);
            if (st) break;
        }
    }
    if (st == DC_OK) {
        if (traj) adj_add_ext(c->gx, traj, c->d_int2ext, m, c->layout, s);
        RET(store_vec(c, c->gx, dL_dx0, host_io));
        RET(store_vec(c, c->gv, dL_dv0, host_io));
        // [B][4] accumulator -> [B][3] output
        const bool dev = is_device_ptr(dL_dparams);
        CK(cudaMemcpy2DAsync(dL_dparams, 3 * sizeof(double), c->dparam_acc, 4 * sizeof(double), 3 * sizeof(double),
                             B, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        host_io |= !dev;
    }
    CK(ctx_sync(c, s));
    if (c->stream2) CK(ctx_sync(c, c->stream2));
    free_pool(c, tmp);
    CK(cudaGetLastError());
    if (st) return st;
    RET(check_device_flags(c));
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
    if (host_io) CK(ctx_sync(c, c->stream));
    return DC_OK;
}

dc_status dc_debug_sweep_wait_timeout(dc_ctx* c, int32_t skip_items) {
    if (!c) return DC_ERR_INVALID;
    if (!c->have_params || c->dm.solver != 1 || !c->dm.ps.tree) {
        c->err = "dc_debug_sweep_wait_timeout: needs global_solver 1 with tree-scheduled sweeps";
        return DC_ERR_INVALID;
    }
    if (skip_items < 1 || skip_items >= c->dm.ps.n_items) {
        c->err = "dc_debug_sweep_wait_timeout: skip_items outside [1, " + std::to_string(c->dm.ps.n_items) + ")";
        return DC_ERR_INVALID;
    }
    launch_solve_fwd_skip(c->dm, c->b, c->y, skip_items, c->stream);
    CK(ctx_sync(c, c->stream));
    CK(cudaGetLastError());
    return check_device_flags(c);
}

dc_status dc_get_instance_nonconverged(dc_ctx* c, int64_t* counts) {
    if (!c || !counts) return DC_ERR_INVALID;
    for (int i = 0; i < c->B; ++i) counts[i] = i < (int)c->inst_noncv.size() ? (int64_t)c->inst_noncv[i] : 0;
    return DC_OK;
}

dc_status dc_debug_front_factor(int32_t n, int32_t p, const float* A, float* out, float* linv_out,
                                int32_t threads, int32_t use_tc, int32_t use_gscr) {
    std::string err;
    const dc_status st = frontal_debug_factor(n, p, A, out, linv_out, threads, use_tc, use_gscr, &err);
    if (st != DC_OK) g_create_err = err;
    return st;
}

dc_status dc_get_stats(dc_ctx* c, dc_stats* o) {
    if (!c || !o) return DC_ERR_INVALID;
    CK(ctx_sync(c, c->stream));
    unsigned long long cnt[3] = {0, 0, 0};
    CK(cudaMemcpyAsync(cnt, c->counters, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
    CK(ctx_sync(c, c->stream));
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
    o->factor_nnz = c->factor_nnz;
    o->solve_nnz = c->fwd_nnz + c->bwd_nnz;
    o->n_free = c->hm.m_free;
    o->nd_levels = c->hm.nd_depth + 1;
    c->kt.flush();
    c->kt2.flush();
    o->kernel_launches = dc_launch_count();
    o->timer_ms = c->kt.ms + c->kt2.ms;
    o->timer_launches = c->kt.launches + c->kt2.launches;
    o->fwd_solve_nnz = c->fwd_nnz;
    o->bwd_solve_nnz = c->bwd_nnz;
    o->front_flops = c->front_flops;
    o->front_levels = c->nlev;
    o->n_supernodes = c->fr.S;
    o->factorisations = c->n_factorisations;
    o->n_instances = c->B;
    o->graphs = c->use_graphs ? 1 : 0;
    o->graph_replays = c->graph_replays;
    o->block_local = c->dm.bs_local;
    o->block_gather = c->dm.bs_gather;
    o->block_node = c->dm.bs_node;
    o->block_elem = c->dm.bs_elem;
    o->adj_batch_iters = c->adj_batch_iters;
    o->global_solver = c->dm.solver;
    o->psolve_flops = c->psolve_flops;
    o->adj_fallbacks = c->adj_fallbacks;
    o->adj_fallback_iters = c->adj_fallback_iters;
    o->layout = c->layout;
    o->contact_compliance = c->prm.contact_compliance;
    o->device_bytes = (int64_t)c->dev_bytes;
    o->device_bytes_peak = (int64_t)c->dev_peak;
    o->n_nodes = c->hm.m;
    o->n_tris = c->hm.T;
    o->bend_nnz = (int64_t)c->hm.bidx.size();
    o->front_entries = (int64_t)c->fr.pool_size;
    return check_device_flags(c);
}

dc_status dc_set_kernel_timer(dc_ctx* c, int32_t kernel_class) {
    if (!c) return DC_ERR_INVALID;
    if (kernel_class < DC_KT_NONE || kernel_class > DC_KT_SWEEPS) {
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
    CK(ctx_sync(c, c->stream));
    CK(cudaGetLastError());
    return check_device_flags(c);
}

void dc_destroy(dc_ctx* c) {
    if (!c) return;
    ctx_sync(c, c->stream);
    if (c->stream2) ctx_sync(c, c->stream2);
    c->kt.release();
    c->kt2.release();
    for (int k = 0; k < 2; ++k) {
        if (c->ev_fact[k]) cudaEventDestroy(c->ev_fact[k]);
        if (c->ev_free[k]) cudaEventDestroy(c->ev_free[k]);
    }
    if (c->ev_seg) cudaEventDestroy(c->ev_seg);
    if (c->stream2) cudaStreamDestroy(c->stream2);
    GraphCache* gcs[] = {&c->g_roll, &c->g_seg[0], &c->g_seg[1]};
    for (GraphCache* g : gcs)
        if (g->exec) cudaGraphExecDestroy(g->exec);
    free_pool(c, c->adj_allocs);
    free_pool(c, c->seg_allocs);
    free_pool(c, c->rec_allocs);
    free_pool(c, c->ck_allocs);
    free_pool(c, c->work_allocs);
    free_pool(c, c->factor_allocs);
    free_pool(c, c->front_allocs);
    free_pool(c, c->mesh_allocs);
    if (c->hpin && !c->hpin_external) cudaFreeHost(c->hpin);
    if (c->h_act_sn) cudaFreeHost(c->h_act_sn);
    if (c->h_act_ch) cudaFreeHost(c->h_act_ch);
    if (c->async_alloc) ctx_sync(c, c->stream);   // the stream-ordered frees above
    if (c->ev_block) cudaEventDestroy(c->ev_block);   // after the last wait on it
    delete c;
}

const char* dc_last_error(dc_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

}  // extern "C"

// Read-only accessors used by dc_static_solve.cu.
bool dc_ctx_ready(const dc_ctx* c) { return c->have_params; }
const DevMesh& dc_ctx_mesh(const dc_ctx* c) { return c->dm; }
const DevParams& dc_ctx_params(const dc_ctx* c) { return c->dp; }
int dc_ctx_device(const dc_ctx* c) { return c->device; }
int dc_ctx_layout(const dc_ctx* c) { return c->layout; }
const int* dc_ctx_int2ext(const dc_ctx* c) { return c->d_int2ext; }
cudaStream_t dc_ctx_stream(const dc_ctx* c) { return c->stream; }
void dc_ctx_set_error(dc_ctx* c, const std::string& msg) { c->err = msg; }
