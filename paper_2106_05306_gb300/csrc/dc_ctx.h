// The context behind the C ABI: one or more cloth instances packed into one
// disconnected problem, their device data, and the work buffers of the forward
// rollout and the checkpointed adjoint.  Shared by dc_api.cu (entry points,
// setup) and dc_driver.cu (time stepping, adjoint Krylov solve, graphs, tuning).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <string>
#include <vector>

#include "dc_adjoint.h"
#include "dc_internal.h"

// Contact record of one forward step, kept for its adjoint step.
struct StepRec {
    int* contact = nullptr;
    int* case_ = nullptr;
    d4* nb = nullptr;
    d4* f = nullptr;
};

// Device allocations of one kind and their total size.
struct Pool {
    std::vector<void*> ptrs;
    size_t bytes = 0;
};

// One captured CUDA graph and what it was captured for.
struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    int ka = -1, kb = -1;
    long long epoch = -1;
    long long launches = 0;        // kernels in the graph
};

// Per-instance state of the batched flexible GMRES.
struct GState {
    double beta0 = 0.0, res = 0.0, prev = 0.0;
    int total = 0, used = 0;
    bool fin = false;              // converged, stagnated or capped: no more work
    bool act = false;              // still iterating in the current restart cycle
};

struct dc_ctx {
    cudaStream_t stream = nullptr;
    int device = 0;                // device current at creation
    int layout = DC_LAYOUT_NODE_MAJOR;   // node arrays at the boundary (dc_set_layout)
    std::string err;
    KTimer kt;
    double front_flops = 0.0;
    double psolve_flops = 0.0;     // one supernodal sweep, 3 columns
    // instances
    int B = 1;
    std::vector<HostMesh> ihm;     // per-instance meshes (refactorised on new parameters)
    std::vector<InstInfo> inst;
    std::vector<dc_params> iprm;   // per-instance normalised parameters
    HostMesh hm;                   // all instances, merged
    HostFactor hf;                 // merged explicit-inverse rows
    long long factor_nnz = 0, fwd_nnz = 0, bwd_nnz = 0;   // scalar factor, L^-1 rows, L^-T rows
    bool have_params = false;
    dc_params prm{};               // the batch-wide fields (and instance 0's material)
    DevParams dp{};
    DevMesh dm{};
    Segs sg{};
    std::vector<int> h_cptr;       // host copy of sg.cptr
    Pool mesh_allocs, factor_allocs, work_allocs, ck_allocs, seg_allocs, adj_allocs, front_allocs;
    bool async_alloc = false;      // stream-ordered allocation on `stream` (contexts of the request server)
    bool blocking_sync = false;    // waits block the thread instead of spinning (contexts of the request server)
    cudaEvent_t ev_block = nullptr;
    size_t dev_bytes = 0, dev_peak = 0;   // device bytes held now / at most
    HostFronts fr;
    FrontDev fdv{};
    int nlev = 0;
    std::vector<int> lvl_maxf;     // largest front of every level
    std::vector<int> lvl_maxp;     // largest pivot block of every level
    std::vector<int> lvl_maxfs;    // ... in nodes (supernodal substitution)
    std::vector<int> ps_lvl_ptr, ps_nbig, ps_nsmall, ps_maxbig;   // supernodal level lists (large, then small)
    int* d_int2ext = nullptr;
    // forward work
    d4 *xa = nullptr, *va = nullptr, *xb = nullptr, *vb = nullptr, *v = nullptr, *b = nullptr, *y = nullptr;
    d4 *c1 = nullptr, *c2 = nullptr, *bu = nullptr, *ind = nullptr;
    double* cc = nullptr;
    StepRec scratch;
    double* stage = nullptr;       // [m][3] staging for host/device conversion
    double* stage2 = nullptr;
    // [0..2] contact cases, [3] sticky fault word of the bounded waits,
    // [4] non-finite forward state, [5] non-positive pivot of the GPU factorisation
    unsigned long long* counters = nullptr;
    // rollout checkpoints
    int ck_n_steps = -1, ck_every = 1, ck_cap = 0;
    d4* ck = nullptr;              // [(cap)][2][m]
    // with checkpoint_every == 1 the rollout keeps every step's contact record, and
    // the backward reads states and records directly (no recomputation)
    std::vector<StepRec> rec_all;
    Pool rec_allocs;
    int rec_cap = 0;
    // backward segment buffers
    int seg_cap = 0;
    d4* segX = nullptr;            // [(cap+1)][m]
    d4* segV = nullptr;
    std::vector<StepRec> seg_rec;
    // adjoint buffers
    int adj_restart_cap = 0;
    AdjDev ad{};                   // the slot in use by the GMRES of the current adjoint step
    AdjDev ads[2]{};               // per-step adjoint data, two slots (even / odd steps)
    FrontDev fds[2]{};             // numeric fronts, two slots
    cudaStream_t stream2 = nullptr;   // assembles and factorises the next step's fronts
    cudaEvent_t ev_fact[2]{}, ev_free[2]{}, ev_seg = nullptr;
    KTimer kt2;
    d4 *gx = nullptr, *gv = nullptr, *gx2 = nullptr, *gv2 = nullptr, *g = nullptr, *rhs = nullptr, *z = nullptr;
    d4 *x1 = nullptr, *r1 = nullptr, *x2 = nullptr, *r2 = nullptr, *ytmp = nullptr, *wv = nullptr, *E = nullptr;
    d4* resid = nullptr;
    double *V = nullptr, *Zb = nullptr, *dcoef = nullptr, *dcoef2 = nullptr, *dnorm = nullptr, *partial = nullptr;
    double *dscale = nullptr, *dparam_acc = nullptr, *dparam_part = nullptr;
    double* hpin = nullptr;        // pinned host scratch
    size_t hpin_cap = 0;           // doubles
    bool hpin_external = false;    // hpin belongs to the caller (a server slot)
    std::vector<GState> gs;
    // fronts and reduction chunks of the instances still iterating (batches):
    // level l's fronts are act_sn[act_ptr[l] .. act_ptr[l+1]); rebuilt when the
    // active set has shrunk by a quarter (the mask keeps results exact between)
    std::vector<int> lvl_inst_ptr;  // [nlev][B + 1]: instance i's fronts in level l start at this lvl_sn index
    // with tree-scheduled solves d_act_sn instead holds the active instances'
    // fronts in the tree order (tq_h filtered), n_act_tq of them
    std::vector<int> tq_h, sn_inst_h;   // fronts in tree order; instance of each front
    int n_act_tq = 0;
    int* d_act_sn = nullptr;
    int* h_act_sn = nullptr;        // pinned
    int* d_act_ch = nullptr;
    int* h_act_ch = nullptr;        // pinned
    int n_act_ch = 0;
    std::vector<int> act_ptr;
    bool act_on = false;
    int act_built = 0;
    // CUDA graphs
    bool use_graphs = false;
    long long graph_epoch = 0;     // bumped whenever a captured pointer or launch shape may change
    long long graph_replays = 0;
    GraphCache g_roll, g_seg[2];
    // stats
    long long steps = 0, adj_steps = 0, adj_iters = 0, adj_max_seen = 0, adj_noncv = 0;
    std::vector<long long> inst_noncv;   // per instance: adjoint steps stopped above adj_tol
    double adj_last_res = 0.0;
    long long n_factorisations = 0;
    long long adj_batch_iters = 0;
    long long adj_fallbacks = 0, adj_fallback_iters = 0;
    // obstacle meshes (dc_add_obstacle_mesh): triangle records, and per mesh its
    // first record and triangle count
    // per-instance step counts (dc_set_instance_steps): device copy, or null
    int* d_inst_steps = nullptr;
    int* d_inst_steps_buf = nullptr;
    std::vector<int> inst_steps;
    std::vector<d4> mesh_rec;      // DC_MESH_REC records per triangle (dc_obstacle.cuh)
    std::vector<int> mesh_t0, mesh_nt;
};

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            c->err = std::string("CUDA error: ") + cudaGetErrorString(e_) + " at " #call;     \
            return (e_ == cudaErrorMemoryAllocation) ? DC_ERR_OOM : DC_ERR_CUDA;              \
        }                                                                                     \
    } while (0)

#define RET(x)                      \
    do {                            \
        dc_status s_ = (x);         \
        if (s_ != DC_OK) return s_; \
    } while (0)

// Waits for the work queued on s so far.  With blocking_sync the thread sleeps
// on an event created with cudaEventBlockingSync instead of spinning, so that
// the request server's many slot threads leave the host's cores to the threads
// preparing the next requests.
inline cudaError_t ctx_sync(dc_ctx* c, cudaStream_t s) {
    if (!c->blocking_sync) return cudaStreamSynchronize(s);
    if (!c->ev_block) {
        cudaError_t e = cudaEventCreateWithFlags(&c->ev_block, cudaEventBlockingSync | cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaEventRecord(c->ev_block, s);
    return e != cudaSuccess ? e : cudaEventSynchronize(c->ev_block);
}

// Allocates count T's (zeroed unless zero = false) into pool.  With
// async_alloc the memory comes from the device's stream-ordered pool on the
// context's stream, so that a context being set up does not synchronise the
// device under other contexts' work.
template <class T>
dc_status dalloc(dc_ctx* c, Pool& pool, T** p, size_t count, bool zero = true) {
    void* q = nullptr;
    size_t bytes = std::max<size_t>(count * sizeof(T), 32);
    cudaError_t e = c->async_alloc ? cudaMallocAsync(&q, bytes, c->stream) : cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        c->err = std::string("device allocation of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e);
        return DC_ERR_OOM;
    }
    if (zero) {
        e = c->async_alloc ? cudaMemsetAsync(q, 0, bytes, c->stream) : cudaMemset(q, 0, bytes);
        if (e != cudaSuccess) {
            c->err = std::string("cudaMemset: ") + cudaGetErrorString(e);
            return DC_ERR_CUDA;
        }
    }
    pool.ptrs.push_back(q);
    pool.bytes += bytes;
    c->dev_bytes += bytes;
    c->dev_peak = std::max(c->dev_peak, c->dev_bytes);
    *p = reinterpret_cast<T*>(q);
    return DC_OK;
}

template <class T>
dc_status upload(dc_ctx* c, Pool& pool, T** p, const std::vector<T>& h) {
    dc_status s = dalloc(c, pool, p, h.size(), false);
    if (s) return s;
    if (!h.empty()) {
        if (c->async_alloc) {
            // h is pageable and may die after the return: wait for the copy
            CK(cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
            CK(ctx_sync(c, c->stream));
        } else {
            CK(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
        }
    }
    return DC_OK;
}

inline void free_pool(dc_ctx* c, Pool& pool) {
    for (void* p : pool.ptrs) {
        if (c->async_alloc)
            cudaFreeAsync(p, c->stream);
        else
            cudaFree(p);
    }
    c->dev_bytes -= std::min(c->dev_bytes, pool.bytes);
    pool.ptrs.clear();
    pool.bytes = 0;
}

// Host-side results of context setup, computed without touching the device (so
// that a request server can prepare requests on host threads while the GPU runs
// others), then uploaded by upload_mesh / upload_params.
struct MeshPrep {
    std::vector<int4> tri4, chunks, pchunks;
    std::vector<d4> G4, qr;
    std::vector<int> iptr, iidx, tbptr, tbidx, node_inst, cptr, pcptr;
    std::vector<double> tbval;
};
struct ParamPrep {
    std::vector<dc_params> q;
    HostFactor hfm;
    HostFronts frm;
    std::vector<double> mass, wt, wb, node_mu, oprm;
    std::vector<int> optr, okind, long_rows, short_rows;
    std::vector<float> tau;
    HostPSolve ps;                 // global_solver 1
    std::vector<double> ccon;      // [m_free] constant compliance (modes other than ROWSUM)
    double front_flops = 0.0;
    long long factor_nnz = 0;
};
// Merges c->ihm into c->hm and builds the device arrays of the mesh.
void prep_mesh_host(dc_ctx* c, MeshPrep& mp);
dc_status upload_mesh(dc_ctx* c, MeshPrep& mp);
// Validates q, factorises every instance's P and builds its fronts (host threads).
dc_status prep_params_host(dc_ctx* c, std::vector<dc_params> q, ParamPrep& pp);
dc_status upload_params(dc_ctx* c, ParamPrep& pp);
// True when two parameter sets may be instances of one batch (equal shared fields).
bool dc_same_batch_fields(const dc_params& a, const dc_params& b);
// Upper bound of the device bytes a context holds through dc_rollout(n_steps) and
// dc_backward (with mesh and parameters prepared).
size_t estimate_device_bytes(const dc_ctx* c, const MeshPrep& mp, const ParamPrep& pp, int n_steps);

// Runs f(0 .. n-1) on up to hardware_concurrency host threads.
void dc_parallel_for(int n, const std::function<void(int)>& f);
bool is_device_ptr(const void* p);
dc_status alloc_rec(dc_ctx* c, Pool& pool, StepRec& r);
dc_status load_vec(dc_ctx* c, const double* ext, d4* out, bool& host_io);
dc_status store_vec(dc_ctx* c, const d4* in, double* ext, bool& host_io);
// One time step (Sec. 3.2) on internal vectors; writes the contact record into r.
// step: the step's index in its rollout; instances whose own step count
// (dc_set_instance_steps) is reached keep their state (-1: no such check).
// step: the index of the step in its rollout (-1: none), for the per-instance step
// counts; plus *step_base when step_base is given (a segment graph replayed for
// several segments reads its first step from device memory).
void run_step(dc_ctx* c, const d4* xin, const d4* vin, d4* xout, d4* vout, StepRec& r, bool count = true,
              int step = -1, const int* step_base = nullptr);
// run_step for steps [0, n) of dc_rollout (graph-captured when enabled)
dc_status rollout_steps(dc_ctx* c, int n_steps, int k);
dc_status ensure_checkpoints(dc_ctx* c, int n_ck);
dc_status ensure_segment(dc_ctx* c, int k);
dc_status ensure_adjoint(dc_ctx* c);
// Recomputes steps [s0, s1) from the checkpoint into the segment buffers.
dc_status recompute_segment(dc_ctx* c, int seg, int s0, int s1);
dc_status ensure_records(dc_ctx* c, int n_steps);
// Per-step adjoint data of the step with record r, ending at (x1, v1), into slot k.
void prepare_step(dc_ctx* c, const StepRec& r, const d4* x1, const d4* v1, int k, cudaStream_t s);
// step: the index of the step being differentiated (for per-instance step counts)
dc_status adjoint_step(dc_ctx* c, const d4* x_n, const d4* x1, const d4* v1, int k, bool& noncv, int step);
dc_status autotune(dc_ctx* c);
// Numeric Cholesky of P on the GPU into the supernodal panels (factor_on_gpu);
// synchronous, DC_ERR_NOT_SPD for a pivot <= 0.
dc_status gpu_factor_P(dc_ctx* c, const HostFronts& frm, double h);
// Reads the device-side error words (bounded-wait timeout, non-finite state);
// synchronises the context's stream.
dc_status check_device_flags(dc_ctx* c);
