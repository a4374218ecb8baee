// solve_static.cu -- mpm_solve_static: the Newton-system solve of mpm_solve
// with its scratch memory in a fixed, library-owned device array instead of a
// caller workspace, for callers that cannot allocate device memory.
//
// The scratch is a file-scope __device__ array of kStaticScratchBytes (64 MiB)
// that every GPU which loads this library holds until the process exits.  In
// host code the array's name is only a host-side stand-in, so its device
// address is looked up once per device with cudaGetSymbolAddress (with that
// device current) and passed to the kernels.
#include <mutex>

#include "mpm_internal.cuh"

namespace mpm {

constexpr size_t kStaticScratchBytes = 64ull << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void* g_static_addr[kMaxDevices];

// Device address of the scratch on the current device (looked up on first use).
static mpm_status static_scratch(void** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return fail(MPM_ERR_CUDA, "mpm_solve_static: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return fail(MPM_ERR_INVALID_ARG, "mpm_solve_static: device %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(MPM_ERR_CUDA, "mpm_solve_static: cudaGetSymbolAddress: %s",
                        cudaGetErrorString(e));
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return MPM_OK;
}

}  // namespace mpm

using namespace mpm;

extern "C" mpm_status mpm_solve_static(const mpm_problem* problem, const mpm_opts* opts,
                                       const float* h, const float* w, const float* g,
                                       const float* y, float* delta, double* resid,
                                       void* stream)
{
    mpm_status s = check_problem(problem);
    if (s != MPM_OK) return s;
    if ((s = check_opts(opts)) != MPM_OK) return s;
    const DevProblem P = make_dev(problem);
    cudaStream_t st = (cudaStream_t)stream;
    if (P.N == 0) {
        if (resid) {
            if ((s = check_dev(resid, "resid", false, 8)) != MPM_OK) return s;
            cudaError_t e = cudaMemsetAsync(resid, 0, sizeof(double), st);
            if (e != cudaSuccess) return fail(MPM_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
        }
        return MPM_OK;
    }
    const size_t need = kHeaderBytes + kPartialBytes + solve_ws_bytes(P);
    if (need > kStaticScratchBytes)
        return fail(MPM_ERR_WORKSPACE_TOO_SMALL,
                    "mpm_solve_static: this problem needs %zu bytes of scratch but the fixed "
                    "scratch holds %zu (about %lld voxels with %d maps); use mpm_solve with a "
                    "caller workspace",
                    need, kStaticScratchBytes,
                    (long long)((kStaticScratchBytes - kHeaderBytes - kPartialBytes) /
                                (solve_ws_bytes(P) / (P.N > 0 ? P.N : 1))),
                    P.K);
    if ((s = check_dev(h, "h", false, 4)) != MPM_OK) return s;
    if ((s = check_dev(w, "w", false, 4)) != MPM_OK) return s;
    if ((s = check_dev(g, "g", false, 4)) != MPM_OK) return s;
    if ((s = check_dev(y, "y", false, 4)) != MPM_OK) return s;
    if ((s = check_dev(delta, "delta", false, 4)) != MPM_OK) return s;
    if ((s = check_dev(resid, "resid", true, 8)) != MPM_OK) return s;
    void* base = nullptr;
    if ((s = static_scratch(&base)) != MPM_OK) return s;
    char* c = static_cast<char*>(base);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(c);
    Reduce red;
    red.partials = reinterpret_cast<double*>(c + kHeaderBytes);
    red.counter = &hdr->counter;
    void* solve = c + kHeaderBytes + kPartialBytes;
    // The scratch keeps the previous call's contents: the status word and the
    // reduction arrival counter must start at zero.
    cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st);
    if (e != cudaSuccess) return fail(MPM_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    e = launch_solve(P, solve_opts(*opts), h, w, g, y, delta, nullptr, resid, nullptr,
                     nullptr, solve, hdr, red, st);
    if (e != cudaSuccess) return fail(MPM_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
    return MPM_OK;
}
