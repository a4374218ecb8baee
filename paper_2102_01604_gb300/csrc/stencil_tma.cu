// stencil_tma.cu -- q = (H + L) p with TMA plane staging (sm_103a).
//
// Same operator as k_pcg_matvec (stencil_kernels.cu): per voxel
//   q_k = sum_j H_kj p_j + lambda_k sum_{m in N(n)} (w_n + w_m)(p_k[n] - p_k[m]) / h^2,
// but every operand reaches shared memory through the tensor memory
// accelerator.  For a tile of TX x TY voxels and each z plane, one thread
// issues bulk tensor copies
//   p  box (TX+8) x (TY+2) x 1 x K  at (x0 - 4, y0 - 1, z, 0)   (tile plus x / y halo)
//   w  box (TX+8) x (TY+2) x 1      at (x0 - 4, y0 - 1, z)
//   H  box TX x TY x 1 x T          at (x0, y0, z, 0)           (only planes computed)
// into two rings: p / w planes (kStagesPW deep; plane z needs z - 1, z and
// z + 1) and H planes (kStagesH deep; plane z needs only its own).  A
// producer warp issues the copies; a stage is refilled as soon as the eight
// compute warps have released it, so both streams run two planes ahead of
// the compute and no compute thread holds loads in registers.  The depth is
// what sets the speed: the copies in flight per SM have to cover the loaded
// DRAM latency.  x coordinates are multiples of 4 floats (16 bytes); boxes
// that leave the volume are zero-filled by the copy engine and masked by the
// boundary flags.  Every mbarrier wait is bounded: on timeout the block
// records kStatusTimeout, stops computing, drains its outstanding copies
// (bounded again) and still takes part in the grid reduction.
#include <cudaTypedefs.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "mpm_internal.cuh"

namespace mpm {

constexpr int kStagesPW = 5;                   // p / w ring
constexpr int kStagesH = 3;                    // H ring
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
    // p / w stage: p then w; H stages follow the p / w ring
    static constexpr int P_OFF = 0;
    static constexpr int W_OFF = align128(P_FLOATS * 4);
    static constexpr int PW_STAGE = W_OFF + align128(W_FLOATS * 4);
    static constexpr int H_STAGE = align128(H_FLOATS * 4);
    static constexpr int H_BASE = kStagesPW * PW_STAGE;
    static constexpr int P_BYTES = P_FLOATS * 4, W_BYTES = W_FLOATS * 4, H_BYTES = H_FLOATS * 4;
    static constexpr int SMEM = H_BASE + kStagesH * H_STAGE + 128;   // + alignment slack
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

// One try: the thread may be suspended until the phase completes or about
// 20 us pass (the suspend-time hint), so waiting warps do not spin on issue
// slots the compute warps need.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(20000u)
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

// Work split: the launch is one wave of resident blocks.  The volume is cut
// into items -- one tile column over one of `nchunk` z ranges -- numbered
// i = chunk * tiles + tile, and block b takes items b, b + G, b + 2G, ...
// (G = gridDim.x), so the blocks running at one time cover neighbouring
// tiles of the same z ranges (their DRAM rows and halos are shared).  The
// ring and its phases run on from one item to the next, so the copies of the
// next item overlap the end of the current one.
template <int K, int TX, int TY>
__global__ void __launch_bounds__(kTmaThreads) k_pcg_matvec_tma(
    DevProblem P, int nchunk, int k_it, const __grid_constant__ CUtensorMap tp,
    const __grid_constant__ CUtensorMap tw, const __grid_constant__ CUtensorMap th,
    float* __restrict__ qout, WsHeader* hdr, Reduce red)
{
    using L = TmaLayout<K, TX, TY>;
    constexpr int kTmaBoxX = L::BX, kTmaBoxY = L::BY, kTmaTX = TX, kTmaTY = TY;
    static_assert(TX * TY == kTmaVoxels, "one compute thread per voxel");
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t pw_full[kStagesPW], pw_empty[kStagesPW];
    __shared__ __align__(8) uint64_t h_full[kStagesH], h_empty[kStagesH];
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
    const int gx = (nx + TX - 1) / TX;
    const int tiles = gx * ((ny + TY - 1) / TY);
    const int items = tiles * nchunk;

    if (tid == 0) {
        s_done = hdr->sc.done;
        s_fail = 0;
        for (int s = 0; s < kStagesPW; ++s) {
            mbar_init(smem_u32(&pw_full[s]), 1);
            mbar_init(smem_u32(&pw_empty[s]), kConsumerWarps);
        }
        for (int s = 0; s < kStagesH; ++s) {
            mbar_init(smem_u32(&h_full[s]), 1);
            mbar_init(smem_u32(&h_empty[s]), kConsumerWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool done = s_done != 0;

    // Load counters: c over the p / w planes this block loads, e over its H
    // planes (one per computed plane), both in order -> ring stage and phase.
    auto pw_stage = [](int c) { return (int)((unsigned)c % (unsigned)kStagesPW); };
    auto pw_phase = [](int c) { return (uint32_t)(((unsigned)c / (unsigned)kStagesPW) & 1u); };
    auto h_stage = [](int e) { return (int)((unsigned)e % (unsigned)kStagesH); };
    auto h_phase = [](int e) { return (uint32_t)(((unsigned)e / (unsigned)kStagesH) & 1u); };
    auto pw_ptr = [&](int c) { return smem + pw_stage(c) * L::PW_STAGE; };

    Acc pq;
    int pw_issued = -1, h_issued = -1;  // last counters issued (producer lane 0)
    if (!done && producer) {
        if (lane == 0) {
            int cb = 0, eb = 0;         // counters of the item's first planes
            for (int i = blockIdx.x; i < items && !s_fail; i += gridDim.x) {
                const int t = i % tiles, ch = i / tiles;
                const int za = (int)((long long)ch * nz / nchunk), zb = (int)((long long)(ch + 1) * nz / nchunk);
                const int x0 = (t % gx) * kTmaTX, y0 = (t / gx) * kTmaTY;
                const int ja = max(za - 1, 0), jb = min(zb, nz - 1);
                for (int j = ja; j <= jb && !s_fail; ++j) {
                    // p / w plane j; its stage must be released by every compute warp
                    const int c = cb + (j - ja);
                    const int s = pw_stage(c);
                    if (c >= kStagesPW && !mbar_wait(smem_u32(&pw_empty[s]), pw_phase(c - kStagesPW))) {
                        s_fail = 1;
                        break;
                    }
                    unsigned char* st = smem + s * L::PW_STAGE;
                    const uint32_t bar = smem_u32(&pw_full[s]);
                    mbar_expect_tx(bar, L::P_BYTES + L::W_BYTES);
                    tma_load_4d(smem_u32(st + L::P_OFF), &tp, x0 - 4, y0 - 1, j, 0, bar);
                    tma_load_3d(smem_u32(st + L::W_OFF), &tw, x0 - 4, y0 - 1, j, bar);
                    pw_issued = c;
                    if (j < za || j >= zb) continue;
                    // H plane j
                    const int e = eb + (j - za);
                    const int sh = h_stage(e);
                    if (e >= kStagesH && !mbar_wait(smem_u32(&h_empty[sh]), h_phase(e - kStagesH))) {
                        s_fail = 1;
                        break;
                    }
                    const uint32_t hbar = smem_u32(&h_full[sh]);
                    mbar_expect_tx(hbar, L::H_BYTES);
                    tma_load_4d(smem_u32(smem + L::H_BASE + sh * L::H_STAGE), &th, x0, y0, j, 0, hbar);
                    h_issued = e;
                }
                cb += jb - ja + 1;
                eb += zb - za;
            }
        }
    } else if (!done) {
        int waited = -1;                // p / w counters [0, waited] are visible to this thread
        int released = 0;               // next p / w counter this warp releases
        int cb = 0, eb = 0;
        for (int i = blockIdx.x; i < items; i += gridDim.x) {
            const int t = i % tiles, ch = i / tiles;
            const int za = (int)((long long)ch * nz / nchunk), zb = (int)((long long)(ch + 1) * nz / nchunk);
            const int x = (t % gx) * kTmaTX + tx, y = (t / gx) * kTmaTY + ty;
            const int ja = max(za - 1, 0), jb = min(zb, nz - 1);
            const bool inside = x < nx && y < ny;
            for (int z = za; z < zb; ++z) {
                const int need = cb + (min(z + 1, nz - 1) - ja);
                const int e = eb + (z - za);
                bool ok = !s_fail;
                for (int c = waited + 1; ok && c <= need; ++c)
                    ok = mbar_wait(smem_u32(&pw_full[pw_stage(c)]), pw_phase(c));
                waited = need;
                if (ok) ok = mbar_wait(smem_u32(&h_full[h_stage(e)]), h_phase(e));
                if (!ok) s_fail = 1;
                if (ok && inside) {
                    const int cz = cb + (z - ja);
                    const float* pcur = reinterpret_cast<const float*>(pw_ptr(cz) + L::P_OFF);
                    const float* wcur = reinterpret_cast<const float*>(pw_ptr(cz) + L::W_OFF);
                    const float* hcur = reinterpret_cast<const float*>(smem + L::H_BASE + h_stage(e) * L::H_STAGE);
                    const int cc = (ty + 1) * kTmaBoxX + tx + 4;      // centre in a p / w plane
                    const bool okxm = x > 0, okxp = x + 1 < nx, okym = y > 0, okyp = y + 1 < ny;
                    const bool okzm = z > 0, okzp = z + 1 < nz;
                    const float* pdn = okzm ? reinterpret_cast<const float*>(pw_ptr(cz - 1) + L::P_OFF) : pcur;
                    const float* wdn = okzm ? reinterpret_cast<const float*>(pw_ptr(cz - 1) + L::W_OFF) : wcur;
                    const float* pup = okzp ? reinterpret_cast<const float*>(pw_ptr(cz + 1) + L::P_OFF) : pcur;
                    const float* wup = okzp ? reinterpret_cast<const float*>(pw_ptr(cz + 1) + L::W_OFF) : wcur;
                    // out-of-volume neighbours: the copy engine zero-fills the
                    // x / y halo and the z neighbour falls back to the centre
                    // plane, so a zero coefficient removes them without a branch
                    const float wc = wcur[cc];
                    const float cxm = okxm ? (wc + wcur[cc - 1]) * P.ihx2 : 0.f;
                    const float cxp = okxp ? (wc + wcur[cc + 1]) * P.ihx2 : 0.f;
                    const float cym = okym ? (wc + wcur[cc - kTmaBoxX]) * P.ihy2 : 0.f;
                    const float cyp = okyp ? (wc + wcur[cc + kTmaBoxX]) * P.ihy2 : 0.f;
                    const float czm = okzm ? (wc + wdn[cc]) * P.ihz2 : 0.f;
                    const float czp = okzp ? (wc + wup[cc]) * P.ihz2 : 0.f;
                    constexpr int PS = kTmaBoxY * kTmaBoxX;             // map stride in a p plane
                    constexpr int HS = kTmaTX * kTmaTY;                 // entry stride in an H plane
                    const int hc = ty * kTmaTX + tx;
                    float hv[L::T];
#pragma unroll
                    for (int m = 0; m < L::T; ++m) hv[m] = hcur[m * HS + hc];
                    float pc[K];
#pragma unroll
                    for (int k = 0; k < K; ++k) pc[k] = pcur[k * PS + cc];
                    float* qn = qout + ((long long)x + (long long)nx * y + (long long)nx * ny * z);
                    float vpq = 0.0f;
#pragma unroll
                    for (int a = 0; a < K; ++a) {
                        const float* pa = pcur + a * PS;
                        const float v = pc[a];
                        float s = cxm * (v - pa[cc - 1]);
                        s += cxp * (v - pa[cc + 1]);
                        s += cym * (v - pa[cc - kTmaBoxX]);
                        s += cyp * (v - pa[cc + kTmaBoxX]);
                        s += czm * (v - pdn[a * PS + cc]);
                        s += czp * (v - pup[a * PS + cc]);
                        float acc = P.lambda[a] * s;
#pragma unroll
                        for (int b = 0; b < K; ++b) acc += hv[a < b ? tri(K, a, b) : tri(K, b, a)] * pc[b];
                        qn[a * N] = acc;
                        vpq += v * acc;
                    }
                    pq.add(vpq);
                }
                // this warp is done with H plane z and no longer needs the p / w
                // planes below z; at the end of the item it releases all of
                // the item's p / w planes
                const int rel_to = z + 1 < zb ? cb + (z - 1 - ja) : cb + (jb - ja);
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(smem_u32(&h_empty[h_stage(e)]));
                    for (int c = released; c <= rel_to; ++c) mbar_arrive(smem_u32(&pw_empty[pw_stage(c)]));
                }
                if (rel_to >= released) released = rel_to + 1;
            }
            cb += jb - ja + 1;
            eb += zb - za;
        }
    }
    __syncthreads();
    if (!done && s_fail) {
        // drain: no copy may still be writing this block's shared memory
        if (producer && lane == 0) {
            // the last fill of each stage (earlier fills have completed before
            // their stage could be refilled)
            for (int c = max(0, pw_issued - kStagesPW + 1); c <= pw_issued; ++c)
                mbar_wait(smem_u32(&pw_full[pw_stage(c)]), pw_phase(c));
            for (int e = max(0, h_issued - kStagesH + 1); e <= h_issued; ++e)
                mbar_wait(smem_u32(&h_full[h_stage(e)]), h_phase(e));
            atomicOr(&hdr->status, kStatusTimeout);
        }
        __syncthreads();
    }
    Acc v[1] = {pq};
    double out[1];
    if (grid_reduce<1>(v, red, out) && tid == 0 && !done) {
        SolveScalars& sc = hdr->sc;
        if (!(out[0] == out[0])) atomicOr(&hdr->status, kStatusNaN);
        if (!(out[0] > 0.0)) {
            sc.done = 1;                 // no further step; the alphas keep their values
        } else {
            sc.alpha_prev = sc.alpha;
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
static cudaError_t launch_tma_k(const DevProblem& P, int nchunk, dim3 grid, const TmaMaps& m, int k_it,
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
        P, nchunk, k_it, m.p[k_it & 1], m.w, m.h, q, hdr, red);
    return cudaGetLastError();
}

template <int K, int TX, int TY>
static int resident_one()
{
    // the occupancy query needs the kernel's shared-memory opt-in first
    int nb = 0;
    if (cudaFuncSetAttribute(k_pcg_matvec_tma<K, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TmaLayout<K, TX, TY>::SMEM) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pcg_matvec_tma<K, TX, TY>, kTmaThreads,
                                                      TmaLayout<K, TX, TY>::SMEM) != cudaSuccess) {
        cudaGetLastError();
        nb = 1;
    }
    return nb > 0 ? nb : 1;
}

// Resident blocks of the TMA matvec per SM for (K, tile) and the SM count of
// the current device, looked up once per device.
static int tma_wave(const DevProblem& P, int tile)
{
    static std::mutex mu;
    static std::map<std::tuple<int, int, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, P.K, tile);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int sms = kNumSm;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = kNumSm;
    }
    int nb;
    if (P.K == 4)
        nb = tile == 1 ? resident_one<4, 32, 8>() : tile == 2 ? resident_one<4, 64, 4>() : resident_one<4, 16, 16>();
    else
        nb = tile == 1 ? resident_one<3, 32, 8>() : tile == 2 ? resident_one<3, 64, 4>() : resident_one<3, 16, 16>();
    return cache[key] = nb * sms;
}

// One wave of resident blocks over tiles x nchunk items (StencilGrid::zc
// carries nchunk, chosen by tma_chunks).
StencilGrid tma_grid(const DevProblem& P, int tile)
{
    const int TX = kTileShapes[tile][0], TY = kTileShapes[tile][1];
    const long long T = (long long)((P.nx + TX - 1) / TX) * ((P.ny + TY - 1) / TY);
    const long long W = tma_wave(P, tile);
    const int best = tma_chunks(T, P.nz, W);
    StencilGrid g;
    g.grid = dim3((unsigned)std::min<long long>(T * best, W), 1, 1);
    g.block = dim3(kTmaThreads, 1, 1);
    g.zc = best;
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
