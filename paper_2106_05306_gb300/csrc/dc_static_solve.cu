// dc_global_solve_static: the global-step solve P_ff^-1 rhs with its scratch
// vectors in a fixed device array instead of memory owned by the context.
//
// Why it exists: some callers may not allocate device memory while they run.
// A serving loop that has handed the rest of HBM to a caching allocator under a
// fixed budget cannot afford an allocation that might fail.  A latency-bound
// control loop cannot afford the device-wide synchronisation that
// cudaMalloc/cudaFree may cause.  This entry point makes no allocation of any
// kind; the caller supplies device input and output arrays, and the three node
// vectors it needs in between live in g_static_scratch below.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds its DC_STATIC_MAX_NODES * 3 * 32 bytes (6 MiB) until the process
// exits.  Host code cannot use the variable's name as a device address; the
// first call on each device looks the address up with cudaGetSymbolAddress
// (that device must be current) and caches it.  Because of that lookup, make
// the first call on a device before any stream capture begins.
//
// All calls share the one array and it keeps whatever the last call left in
// it: each call rewrites every entry it reads (the permuted input, the forward
// result, and the pinned-node rows of the solution, which are zeroed) before
// reading it.  Calls whose execution overlaps on the GPU (different streams or
// contexts on the same device) race on the array; serialise them.  With
// global_solver 1 the supernodal sweeps also write the context's own update
// and solution vectors and dependency flags (allocated once by dc_set_params),
// so calls on one context must also be serialised with its other calls, which
// its stream does.
//
// The scratch address is looked up for the device the context was created on,
// which must be the current device (a kernel on one device must not be handed
// another device's array).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "dc_internal.h"

namespace {

constexpr int DC_STATIC_MAX_NODES = 1 << 16;
constexpr int DC_STATIC_MAX_DEVICES = 64;

static __device__ __align__(256) d4 g_static_scratch[3 * DC_STATIC_MAX_NODES];

std::mutex g_static_mu;
d4* g_static_ptr[DC_STATIC_MAX_DEVICES] = {nullptr};

bool device_accessible(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// Accessors of the context (defined in dc_api.cu).
bool dc_ctx_ready(const dc_ctx* c);
int dc_ctx_device(const dc_ctx* c);
int dc_ctx_layout(const dc_ctx* c);
const DevMesh& dc_ctx_mesh(const dc_ctx* c);
const DevParams& dc_ctx_params(const dc_ctx* c);
const int* dc_ctx_int2ext(const dc_ctx* c);
cudaStream_t dc_ctx_stream(const dc_ctx* c);
void dc_ctx_set_error(dc_ctx* c, const std::string& msg);

extern "C" dc_status dc_global_solve_static(dc_ctx* c, const double* rhs, double* out) {
    if (!c) return DC_ERR_INVALID;
    if (!dc_ctx_ready(c)) {
        dc_ctx_set_error(c, "dc_global_solve_static: call dc_set_params first");
        return DC_ERR_STATE;
    }
    const DevMesh& dm = dc_ctx_mesh(c);
    if (dm.m > DC_STATIC_MAX_NODES) {
        dc_ctx_set_error(c, "dc_global_solve_static: the mesh has " + std::to_string(dm.m) +
                                " nodes; the static scratch serves at most " +
                                std::to_string(DC_STATIC_MAX_NODES));
        return DC_ERR_INVALID;
    }
    if (!rhs || !out || !device_accessible(rhs) || !device_accessible(out)) {
        dc_ctx_set_error(c, "dc_global_solve_static: rhs and out must be device arrays");
        return DC_ERR_INVALID;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= DC_STATIC_MAX_DEVICES) {
        cudaGetLastError();
        dc_ctx_set_error(c, "dc_global_solve_static: no usable current device");
        return DC_ERR_CUDA;
    }
    if (dev != dc_ctx_device(c)) {
        dc_ctx_set_error(c, "dc_global_solve_static: device " + std::to_string(dc_ctx_device(c)) +
                                " (the context's) must be current, not device " + std::to_string(dev));
        return DC_ERR_INVALID;
    }
    d4* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mu);
        if (!g_static_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess) {
                cudaGetLastError();   // do not leave the error for a later call to report
                dc_ctx_set_error(c, std::string("dc_global_solve_static: cudaGetSymbolAddress: ") +
                                        cudaGetErrorString(e));
                return DC_ERR_CUDA;
            }
            g_static_ptr[dev] = static_cast<d4*>(p);
        }
        scratch = g_static_ptr[dev];
    }
    d4* b = scratch;
    d4* y = scratch + DC_STATIC_MAX_NODES;
    d4* v = scratch + 2 * DC_STATIC_MAX_NODES;
    cudaStream_t s = dc_ctx_stream(c);
    const int* int2ext = dc_ctx_int2ext(c);
    launch_permute_in(rhs, b, int2ext, dm.m, dc_ctx_layout(c), s);
    launch_solve_fwd(dm, b, y, s);
    launch_zero_pins(v, dm.m_free, dm.m, s);
    launch_solve_bwd(dm, dc_ctx_params(c), y, v, 0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, s);
    launch_permute_out(v, out, int2ext, dm.m, dc_ctx_layout(c), s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        dc_ctx_set_error(c, std::string("dc_global_solve_static: ") + cudaGetErrorString(e));
        return DC_ERR_CUDA;
    }
    return DC_OK;
}
