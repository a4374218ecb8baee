// stencil_tma.cu -- q = (H + L) p with TMA plane staging (sm_103a).
//
// Same operator as k_pcg_matvec (stencil_kernels.cu): per voxel
//   q_k = sum_j H_kj p_j + lambda_k sum_{m in N(n)} (w_n + w_m)(p_k[n] - p_k[m]) / h^2,
// but every operand reaches shared memory through the tensor memory
// accelerator: for each z plane, one thread issues three bulk tensor copies
//   p  box 24 x 18 x 1 x K  at (x0 - 4, y0 - 1, z, 0)   (tile plus x / y halo)
//   w  box 24 x 18 x 1      at (x0 - 4, y0 - 1, z)
//   H  box 16 x 16 x 1 x T  at (x0, y0, z, 0)           (only planes the block owns)
// into a ring of kStages stage buffers.  A producer warp issues the copies; a
// stage is refilled as soon as the eight compute warps have released it, so
// while a warp computes plane z the copies for planes up to z + 3 can be in
// flight and no compute thread holds loads in registers.  x coordinates are multiples of 4 floats (16 bytes); boxes that
// leave the volume are zero-filled by the copy engine and masked by the
// boundary flags.  Every mbarrier wait is bounded: on timeout the block
// records kStatusTimeout, stops computing, drains its outstanding copies
// (bounded again) and still takes part in the grid reduction.
#include <cudaTypedefs.h>

#include <map>
#include <mutex>
#include <tuple>

#include "mpm_internal.cuh"

namespace mpm {

constexpr int kStages = 4;
constexpr int kTmaVoxels = 256;                // voxels per tile, one compute thread each
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz

// Tile of TX x TY voxels; the p / w boxes add a one-voxel y halo and a
// four-voxel x margin on each side (x0 - 4 keeps the copy 16-byte aligned).
template <int K, int TX, int TY>
struct TmaLayout {
    static constexpr int BX = TX + 8, BY = TY + 2;
    static constexpr int T = K * (K + 1) / 2;
    static constexpr int P_FLOATS = K * BY * BX;
    static constexpr int W_FLOATS = BY * BX;
    static constexpr int H_FLOATS = T * TY * TX;
    static constexpr int align128(int bytes) { return (bytes + 127) / 128 * 128; }
    static constexpr int P_OFF = 0;
    static constexpr int W_OFF = align128(P_FLOATS * 4);
    static constexpr int H_OFF = W_OFF + align128(W_FLOATS * 4);
    static constexpr int STAGE = H_OFF + align128(H_FLOATS * 4);
    static constexpr int P_BYTES = P_FLOATS * 4, W_BYTES = W_FLOATS * 4, H_BYTES = H_FLOATS * 4;
    static constexpr int SMEM = kStages * STAGE + 128;   // + alignment slack
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false after about kWaitCycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Warp-specialised pipeline: warps 0-7 compute one voxel per thread, warp 8
// is the producer.  Per stage, `full` completes when the copies have landed
// and `empty` when all eight compute warps have released the plane; nobody
// waits at a block-wide barrier inside the plane loop.
constexpr int kConsumerWarps = kTmaVoxels / 32;
constexpr int kTmaThreads = kTmaVoxels + 32;

template <int K, int TX, int TY>
__global__ void __launch_bounds__(kTmaThreads) k_pcg_matvec_tma(
    DevProblem P, int zc, int k_it, const __grid_constant__ CUtensorMap tp,
    const __grid_constant__ CUtensorMap tw, const __grid_constant__ CUtensorMap th,
    float* __restrict__ qout, WsHeader* hdr, Reduce red)
{
    using L = TmaLayout<K, TX, TY>;
    constexpr int kTmaBoxX = L::BX, kTmaBoxY = L::BY, kTmaTX = TX, kTmaTY = TY;
    static_assert(TX * TY == kTmaVoxels, "one compute thread per voxel");
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kStages];
    __shared__ __align__(8) uint64_t empty[kStages];
    __shared__ int s_done;
    __shared__ volatile int s_fail;
    unsigned char* smem =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const bool producer = warp == kConsumerWarps;
    const int tx = tid % kTmaTX, ty = tid / kTmaTX;          // meaningful for compute warps
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const long long N = P.N;
    const int x0 = blockIdx.x * kTmaTX, y0 = blockIdx.y * kTmaTY;
    const int z0 = blockIdx.z * zc;
    const int z1 = min(nz, z0 + zc);
    const int j0 = max(z0 - 1, 0);          // first plane this block loads
    const int jmax = min(z1, nz - 1);       // last plane this block loads

    if (tid == 0) {
        s_done = hdr->sc.done;
        s_fail = 0;
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), kConsumerWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool done = s_done != 0;

    auto stage_of = [&](int j) { return (j - j0) % kStages; };
    auto fill_of = [&](int j) { return (j - j0) / kStages; };

    Acc pq;
    int issued_to = j0 - 1;
    if (!done && producer) {
        if (lane == 0) {
            for (int j = j0; j <= jmax; ++j) {
                const int s = stage_of(j), f = fill_of(j);
                // the plane that held this stage must be released by every compute warp
                if (f >= 1 && !mbar_wait(smem_u32(&empty[s]), (uint32_t)((f - 1) & 1))) {
                    s_fail = 1;
                    break;
                }
                if (s_fail) break;
                unsigned char* st = smem + s * L::STAGE;
                const uint32_t bar = smem_u32(&full[s]);
                const bool own = j >= z0 && j < z1;
                mbar_expect_tx(bar, L::P_BYTES + L::W_BYTES + (own ? L::H_BYTES : 0));
                tma_load_4d(smem_u32(st + L::P_OFF), &tp, x0 - 4, y0 - 1, j, 0, bar);
                tma_load_3d(smem_u32(st + L::W_OFF), &tw, x0 - 4, y0 - 1, j, bar);
                if (own) tma_load_4d(smem_u32(st + L::H_OFF), &th, x0, y0, j, 0, bar);
                issued_to = j;
            }
        }
    } else if (!done) {
        const int x = x0 + tx, y = y0 + ty;
        const bool inside = x < nx && y < ny;
        int waited_to = j0 - 1;               // planes [j0, waited_to] are visible to this thread
        for (int z = z0; z < z1; ++z) {
            const int need = min(z + 1, nz - 1);
            bool ok = !s_fail;
            for (int j = waited_to + 1; ok && j <= need; ++j)
                ok = mbar_wait(smem_u32(&full[stage_of(j)]), (uint32_t)(fill_of(j) & 1));
            waited_to = need;
            if (!ok) s_fail = 1;
            if (ok && inside) {
                const float* pcur = reinterpret_cast<const float*>(smem + stage_of(z) * L::STAGE + L::P_OFF);
                const float* wcur = reinterpret_cast<const float*>(smem + stage_of(z) * L::STAGE + L::W_OFF);
                const float* hcur = reinterpret_cast<const float*>(smem + stage_of(z) * L::STAGE + L::H_OFF);
                const int cc = (ty + 1) * kTmaBoxX + tx + 4;      // centre in a p / w plane
                const bool okxm = x > 0, okxp = x + 1 < nx, okym = y > 0, okyp = y + 1 < ny;
                const bool okzm = z > 0, okzp = z + 1 < nz;
                const float* pdn = okzm ? reinterpret_cast<const float*>(smem + stage_of(z - 1) * L::STAGE + L::P_OFF) : pcur;
                const float* wdn = okzm ? reinterpret_cast<const float*>(smem + stage_of(z - 1) * L::STAGE + L::W_OFF) : wcur;
                const float* pup = okzp ? reinterpret_cast<const float*>(smem + stage_of(z + 1) * L::STAGE + L::P_OFF) : pcur;
                const float* wup = okzp ? reinterpret_cast<const float*>(smem + stage_of(z + 1) * L::STAGE + L::W_OFF) : wcur;
                const float wc = wcur[cc];
                const float cxm = okxm ? (wc + wcur[cc - 1]) * P.ihx2 : 0.f;
                const float cxp = okxp ? (wc + wcur[cc + 1]) * P.ihx2 : 0.f;
                const float cym = okym ? (wc + wcur[cc - kTmaBoxX]) * P.ihy2 : 0.f;
                const float cyp = okyp ? (wc + wcur[cc + kTmaBoxX]) * P.ihy2 : 0.f;
                const float czm = okzm ? (wc + wdn[cc]) * P.ihz2 : 0.f;
                const float czp = okzp ? (wc + wup[cc]) * P.ihz2 : 0.f;
                constexpr int PS = kTmaBoxY * kTmaBoxX;             // map stride in a p plane
                float pc[K];
#pragma unroll
                for (int k = 0; k < K; ++k) pc[k] = pcur[k * PS + cc];
                const int hc = ty * kTmaTX + tx;
                const long long n = (long long)x + (long long)nx * y + (long long)nx * ny * z;
                float vpq = 0.0f;
#pragma unroll
                for (int a = 0; a < K; ++a) {
                    const float v = pc[a];
                    const float* pa = pcur + a * PS;
                    float s = 0.f;
                    if (okxm) s += cxm * (v - pa[cc - 1]);
                    if (okxp) s += cxp * (v - pa[cc + 1]);
                    if (okym) s += cym * (v - pa[cc - kTmaBoxX]);
                    if (okyp) s += cyp * (v - pa[cc + kTmaBoxX]);
                    if (okzm) s += czm * (v - pdn[a * PS + cc]);
                    if (okzp) s += czp * (v - pup[a * PS + cc]);
                    float acc = P.lambda[a] * s;
#pragma unroll
                    for (int b = 0; b < K; ++b)
                        acc += hcur[(a < b ? tri(K, a, b) : tri(K, b, a)) * (kTmaTX * kTmaTY) + hc] * pc[b];
                    qout[a * N + n] = acc;
                    vpq += v * acc;
                }
                pq.add(vpq);
            }
            // this warp no longer needs plane z - 1
            if (z - 1 >= j0) {
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&empty[stage_of(z - 1)]));
            }
        }
    }
    __syncthreads();
    if (!done && s_fail) {
        // drain: no copy may still be writing this block's shared memory
        if (producer && lane == 0) {
            // the last fill of each stage (earlier fills have completed before
            // their stage could be refilled)
            for (int j = max(j0, issued_to - kStages + 1); j <= issued_to; ++j)
                mbar_wait(smem_u32(&full[stage_of(j)]), (uint32_t)(fill_of(j) & 1));
            atomicOr(&hdr->status, kStatusTimeout);
        }
        __syncthreads();
    }
    Acc v[1] = {pq};
    double out[1];
    if (grid_reduce<1>(v, red, out) && tid == 0 && !done) {
        SolveScalars& sc = hdr->sc;
        if (k_it > 0) sc.xcount = k_it;
        if (!(out[0] == out[0])) atomicOr(&hdr->status, kStatusNaN);
        if (!(out[0] > 0.0)) {
            sc.done = 1;                 // no further step; alpha keeps the previous value
        } else {
            sc.alpha = sc.rz / out[0];
        }
    }
}

// ------------------------------------------------------------------ host

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

static bool encode(CUtensorMap* m, const float* base, int rank, const cuuint64_t* dims,
                   const cuuint64_t* strides, const cuuint32_t* box)
{
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<float*>(base),
                       dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tile shapes the TMA matvec is compiled for (x by y voxels).
static const int kTileShapes[][2] = {{16, 16}, {32, 8}, {64, 4}};

int tma_tile_count() { return 3; }

// Tile shape per volume: set by the autotuner (mpm_autotune), else a default.
static std::mutex g_tile_mu;
static std::map<std::tuple<int, int, int, int>, int> g_tile_cache;

void tma_tile_set(const DevProblem& P, int tile)
{
    std::lock_guard<std::mutex> lk(g_tile_mu);
    g_tile_cache[std::make_tuple(P.nx, P.ny, P.nz, P.K)] = tile;
}

int tma_tile_choice(const DevProblem& P)
{
    {
        std::lock_guard<std::mutex> lk(g_tile_mu);
        auto it = g_tile_cache.find(std::make_tuple(P.nx, P.ny, P.nz, P.K));
        if (it != g_tile_cache.end()) return it->second;
    }
    return (P.nx >= 40 && P.ny >= 10) ? 1 : 0;    // 32 x 8 when it fits, else 16 x 16
}

bool make_tma_maps(const DevProblem& P, const float* h, const float* w, const float* p0,
                   const float* p1, int tile, TmaMaps* out)
{
    if (tile < 0 || tile >= tma_tile_count()) return false;
    const int TX = kTileShapes[tile][0], TY = kTileShapes[tile][1];
    const int BX = TX + 8, BY = TY + 2;
    // TMA needs 16-byte aligned bases and row strides, and boxes no larger
    // than the volume in x and y.
    if (P.nx % 4 != 0 || P.nx < BX || P.ny < BY) return false;
    if ((reinterpret_cast<uintptr_t>(h) | reinterpret_cast<uintptr_t>(w) |
         reinterpret_cast<uintptr_t>(p0) | reinterpret_cast<uintptr_t>(p1)) % 16)
        return false;
    if (!encode_fn()) return false;
    const cuuint64_t nx = P.nx, ny = P.ny, nz = P.nz;
    const cuuint64_t row = nx * 4, plane = nx * ny * 4, vol = (cuuint64_t)P.N * 4;
    const cuuint64_t dp[4] = {nx, ny, nz, (cuuint64_t)P.K};
    const cuuint64_t dh[4] = {nx, ny, nz, (cuuint64_t)P.T};
    const cuuint64_t s4[3] = {row, plane, vol};
    const cuuint64_t d3[3] = {nx, ny, nz};
    const cuuint64_t s3[2] = {row, plane};
    const cuuint32_t bp[4] = {(cuuint32_t)BX, (cuuint32_t)BY, 1, (cuuint32_t)P.K};
    const cuuint32_t bw[3] = {(cuuint32_t)BX, (cuuint32_t)BY, 1};
    const cuuint32_t bh[4] = {(cuuint32_t)TX, (cuuint32_t)TY, 1, (cuuint32_t)P.T};
    out->tile = tile;
    return encode(&out->p[0], p0, 4, dp, s4, bp) && encode(&out->p[1], p1, 4, dp, s4, bp) &&
           encode(&out->w, w, 3, d3, s3, bw) && encode(&out->h, h, 4, dh, s4, bh);
}

template <int K, int TX, int TY>
static cudaError_t launch_tma_k(const DevProblem& P, int zc, dim3 grid, const TmaMaps& m, int k_it,
                                float* q, WsHeader* hdr, Reduce red, cudaStream_t st)
{
    using L = TmaLayout<K, TX, TY>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_pcg_matvec_tma<K, TX, TY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_pcg_matvec_tma<K, TX, TY><<<grid, dim3(kTmaThreads, 1, 1), L::SMEM, st>>>(
        P, zc, k_it, m.p[k_it & 1], m.w, m.h, q, hdr, red);
    return cudaGetLastError();
}

StencilGrid tma_grid(const DevProblem& P, int tile)
{
    StencilGrid g = stencil_grid(P, kTileShapes[tile][0], kTileShapes[tile][1]);
    g.block = dim3(kTmaThreads, 1, 1);
    return g;
}

template <int K>
static cudaError_t launch_tma_tile(const DevProblem& P, const StencilGrid& g, const TmaMaps& m,
                                   int k_it, float* q, WsHeader* hdr, Reduce red, cudaStream_t st)
{
    switch (m.tile) {
    case 1: return launch_tma_k<K, 32, 8>(P, g.zc, g.grid, m, k_it, q, hdr, red, st);
    case 2: return launch_tma_k<K, 64, 4>(P, g.zc, g.grid, m, k_it, q, hdr, red, st);
    default: return launch_tma_k<K, 16, 16>(P, g.zc, g.grid, m, k_it, q, hdr, red, st);
    }
}

template <int K, int TX, int TY>
static cudaError_t prime_one()
{
    return cudaFuncSetAttribute(k_pcg_matvec_tma<K, TX, TY>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TmaLayout<K, TX, TY>::SMEM);
}

cudaError_t prime_tma_kernels()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = prime_one<4, 16, 16>();
    if (!e) e = prime_one<4, 32, 8>();
    if (!e) e = prime_one<4, 64, 4>();
    if (!e) e = prime_one<3, 16, 16>();
    if (!e) e = prime_one<3, 32, 8>();
    if (!e) e = prime_one<3, 64, 4>();
    if (!e) done = true;
    return e;
}

cudaError_t launch_matvec_tma(const DevProblem& P, const StencilGrid& g, const TmaMaps& m,
                              int k_it, float* q, WsHeader* hdr, Reduce red, cudaStream_t st)
{
    if (P.K == 4) return launch_tma_tile<4>(P, g, m, k_it, q, hdr, red, st);
    return launch_tma_tile<3>(P, g, m, k_it, q, hdr, red, st);
}

}  // namespace mpm
