// stencil_tma.cu -- q = (H + L) p with TMA plane staging (sm_103a).
//
// Same operator as k_pcg_matvec (stencil_kernels.cu): per voxel
//   q_k = sum_j H_kj p_j + lambda_k sum_{m in N(n)} (w_n + w_m)(p_k[n] - p_k[m]) / h^2,
// but every operand reaches shared memory through the tensor memory
// accelerator: for each z plane, one thread issues three bulk tensor copies
//   p  box 24 x 18 x 1 x K  at (x0 - 4, y0 - 1, z, 0)   (tile plus x / y halo)
//   w  box 24 x 18 x 1      at (x0 - 4, y0 - 1, z)
//   H  box 16 x 16 x 1 x T  at (x0, y0, z, 0)           (only planes the block owns)
// into a ring of kStages stage buffers, completing on one mbarrier per stage.
// The block marches up its run of z planes; while it computes plane z the
// copies for planes up to z + 2 are in flight, so no thread holds loads in
// registers.  x coordinates are multiples of 4 floats (16 bytes); boxes that
// leave the volume are zero-filled by the copy engine and masked by the
// boundary flags.  Every mbarrier wait is bounded: on timeout the block
// records kStatusTimeout, stops computing, drains its outstanding copies
// (bounded again) and still takes part in the grid reduction.
#include <cudaTypedefs.h>

#include "mpm_internal.cuh"

namespace mpm {

constexpr int kTmaTX = 16, kTmaTY = 16;        // tile of voxels, one thread each
constexpr int kTmaBoxX = kTmaTX + 8;           // x0 - 4 .. x0 + 19 (16-byte aligned start)
constexpr int kTmaBoxY = kTmaTY + 2;           // y0 - 1 .. y0 + 16
constexpr int kStages = 4;
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz

template <int K>
struct TmaLayout {
    static constexpr int T = K * (K + 1) / 2;
    static constexpr int P_FLOATS = K * kTmaBoxY * kTmaBoxX;
    static constexpr int W_FLOATS = kTmaBoxY * kTmaBoxX;
    static constexpr int H_FLOATS = T * kTmaTY * kTmaTX;
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

template <int K>
__global__ void __launch_bounds__(kTmaTX * kTmaTY) k_pcg_matvec_tma(
    DevProblem P, int zc, int k_it, const __grid_constant__ CUtensorMap tp,
    const __grid_constant__ CUtensorMap tw, const __grid_constant__ CUtensorMap th,
    float* __restrict__ qout, WsHeader* hdr, Reduce red)
{
    using L = TmaLayout<K>;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[kStages];
    __shared__ int s_done, s_fail;
    unsigned char* smem =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = tx + ty * kTmaTX;
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
        for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool done = s_done != 0;

    auto stage_of = [&](int j) { return (j - j0) % kStages; };
    auto parity_of = [&](int j) { return (uint32_t)(((j - j0) / kStages) & 1); };
    auto issue = [&](int j) {                 // one thread: copies for plane j
        const int s = stage_of(j);
        unsigned char* st = smem + s * L::STAGE;
        const uint32_t bar = smem_u32(&bars[s]);
        const bool own = j >= z0 && j < z1;
        mbar_expect_tx(bar, L::P_BYTES + L::W_BYTES + (own ? L::H_BYTES : 0));
        tma_load_4d(smem_u32(st + L::P_OFF), &tp, x0 - 4, y0 - 1, j, 0, bar);
        tma_load_3d(smem_u32(st + L::W_OFF), &tw, x0 - 4, y0 - 1, j, bar);
        if (own) tma_load_4d(smem_u32(st + L::H_OFF), &th, x0, y0, j, 0, bar);
    };

    int issued_to = j0 - 1;                   // last plane issued (thread 0's view)
    if (!done && tid == 0) {
        for (int j = j0; j <= jmax && j < j0 + kStages; ++j) issue(j);
        issued_to = min(jmax, j0 + kStages - 1);
    }

    const int x = x0 + tx, y = y0 + ty;
    const bool inside = x < nx && y < ny;
    Acc pq;
    if (!done) {
        int waited_to = j0 - 1;               // planes [j0, waited_to] are visible to this thread
        for (int z = z0; z < z1; ++z) {
            // make planes z - 1 .. z + 1 visible
            const int need = min(z + 1, nz - 1);
            bool ok = true;
            for (int j = waited_to + 1; j <= need; ++j)
                ok &= mbar_wait(smem_u32(&bars[stage_of(j)]), parity_of(j));
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
            __syncthreads();                  // every thread is done with plane z - 1
            if (s_fail) break;
            if (tid == 0) {
                const int j = z - 1 + kStages;    // refill the stage of plane z - 1
                if (z - 1 >= j0 && j <= jmax) {
                    issue(j);
                    issued_to = j;
                }
            }
        }
        if (s_fail) {
            // drain: no copy may still be writing this block's shared memory
            if (tid == 0) {
                for (int j = j0; j <= issued_to; ++j) mbar_wait(smem_u32(&bars[stage_of(j)]), parity_of(j));
                atomicOr(&hdr->status, kStatusTimeout);
            }
            __syncthreads();
        }
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

bool make_tma_maps(const DevProblem& P, const float* h, const float* w, const float* p0,
                   const float* p1, TmaMaps* out)
{
    // TMA needs 16-byte aligned bases and row strides, and boxes no larger
    // than the volume in x and y.
    if (P.nx % 4 != 0 || P.nx < kTmaBoxX || P.ny < kTmaBoxY) return false;
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
    const cuuint32_t bp[4] = {kTmaBoxX, kTmaBoxY, 1, (cuuint32_t)P.K};
    const cuuint32_t bw[3] = {kTmaBoxX, kTmaBoxY, 1};
    const cuuint32_t bh[4] = {kTmaTX, kTmaTY, 1, (cuuint32_t)P.T};
    return encode(&out->p[0], p0, 4, dp, s4, bp) && encode(&out->p[1], p1, 4, dp, s4, bp) &&
           encode(&out->w, w, 3, d3, s3, bw) && encode(&out->h, h, 4, dh, s4, bh);
}

template <int K>
static cudaError_t launch_tma_k(const DevProblem& P, int zc, dim3 grid, const TmaMaps& m, int k_it,
                                float* q, WsHeader* hdr, Reduce red, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_pcg_matvec_tma<K>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             TmaLayout<K>::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_pcg_matvec_tma<K><<<grid, dim3(kTmaTX, kTmaTY, 1), TmaLayout<K>::SMEM, st>>>(
        P, zc, k_it, m.p[k_it & 1], m.w, m.h, q, hdr, red);
    return cudaGetLastError();
}

StencilGrid tma_grid(const DevProblem& P) { return stencil_grid(P, kTmaTX, kTmaTY); }

cudaError_t launch_matvec_tma(const DevProblem& P, const StencilGrid& g, const TmaMaps& m,
                              int k_it, float* q, WsHeader* hdr, Reduce red, cudaStream_t st)
{
    if (P.K == 4) return launch_tma_k<4>(P, g.zc, g.grid, m, k_it, q, hdr, red, st);
    return launch_tma_k<3>(P, g.zc, g.grid, m, k_it, q, hdr, red, st);
}

}  // namespace mpm
