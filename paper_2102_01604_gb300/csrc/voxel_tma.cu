// voxel_tma.cu -- the fused voxel pass (signal, residuals, gradient and the
// approximate Hessian of Eq. 24, NLL in float64) with its inputs staged in
// shared memory by bulk copies (sm_103a).
//
// The volume is cut into chunks of kChunk consecutive voxels; a chunk needs
// one row of kChunk values from each of its input planes: the K maps, B1+,
// then per contrast its B1- and its echoes, in that order.  A producer warp
// streams these rows, one cp.async.bulk each, into a ring of kSlots row
// slots, running up to a ring ahead of the seven compute warps.  Rows travel
// in groups (the maps with B1+, then each contrast's B1- and echoes, at most
// kGroupMax rows; contrasts with more echoes take the unstaged pass): a
// group's copies complete one full mbarrier, and each compute warp releases
// the group, on its empty mbarrier, once it has read the group's last row.
// So the DRAM reads are always in flight ahead of the arithmetic, whatever the
// occupancy (two blocks per SM at the 128 registers the two-voxel arithmetic
// needs), and a compute thread waits once per group, not once per row.  Each
// compute thread takes two neighbouring voxels of the chunk, with the
// arithmetic of the unstaged pass (voxel_model.cuh) in paired float32
// instructions, so g and h are the same bit for bit.
//
// Every mbarrier wait is bounded: on timeout the block stops waiting, drains
// the copies it issued (bounded again), records kStatusTimeout and still
// takes part in the NLL reduction.
#include <algorithm>

#include "mpm_internal.cuh"
#include "tma_common.cuh"
#include "voxel_model.cuh"

namespace mpm {

constexpr int kGhWarps = 7;                        // compute warps
constexpr int kGhThreads = (kGhWarps + 1) * 32;    // plus the producer warp
constexpr int kChunk = kGhWarps * 32 * 2;          // voxels per chunk: two per compute thread
constexpr int kSlotBytes = kChunk * 4;             // one row of float32 values (1792 B)
constexpr int kSlots = 32;                         // ring of row slots
constexpr int kGhSmem = kSlots * kSlotBytes + 128; // + alignment slack
constexpr int kGroupMax = 16;                      // rows per group: two groups always fit the ring
constexpr int kGroupBars = 8;                      // full / empty mbarrier pairs, one per group in flight
constexpr int kMaxRows = 4 + 1 + MPM_MAX_CONTRASTS + MPM_MAX_IMAGES;
constexpr int kMaxGroups = 1 + MPM_MAX_CONTRASTS;
static_assert(2 * kGroupMax <= kSlots, "a group and the next fit the ring together");
static_assert(kSlotBytes % 128 == 0, "slots stay 128-byte aligned");
static_assert(2 * (kGhSmem + 1024) <= 228 * 1024, "two blocks per SM");

// Two neighbouring values of a row slot in shared memory, as floats.
__device__ __forceinline__ void slot_pair(const float* p, float (&o)[2])
{
    const float2 v = *reinterpret_cast<const float2*>(p);
    o[0] = v.x;
    o[1] = v.y;
}

__device__ __forceinline__ void slot_pair(const __nv_bfloat16* p, float (&o)[2])
{
    const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(p);
    o[0] = __low2float(v);
    o[1] = __high2float(v);
}

template <int K, int PRE, typename XT>
__device__ __forceinline__ void grad_hess_tma_body(const DevProblem& P, const XT* __restrict__ x,
                                                   const float* __restrict__ y,
                                                   const float* __restrict__ b1p,
                                                   const float* __restrict__ b1m, float* __restrict__ g,
                                                   float* __restrict__ h, double* nll, Reduce red,
                                                   unsigned* status, long long wait_cycles, int withhold,
                                                   const VGrid& vg)
{
    constexpr int T = K * (K + 1) / 2;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kGroupBars], empty[kGroupBars];
    __shared__ const unsigned char* s_row_base[kMaxRows];   // plane of each row of a chunk
    __shared__ unsigned char s_row_elem[kMaxRows];           // its element size
    __shared__ unsigned char s_gsize[kMaxGroups];            // rows of each group of a chunk
    __shared__ unsigned short s_gstart[kMaxGroups];          // first row of each group
    __shared__ int s_ngroups;
    __shared__ volatile int s_fail;
    unsigned char* smem =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long N = P.N;
    const long long nchunks = (N + kChunk - 1) / kChunk;

    if (tid == 0) {
        s_fail = 0;
        for (int s = 0; s < kGroupBars; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), kGhWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // The rows of a chunk in the order the compute warps read them, in
        // groups: the maps with B1+, then per contrast its B1- and echoes.
        int r = 0, ng = 0;
        auto add_row = [&](const void* base, int elem) {
            s_row_base[r] = static_cast<const unsigned char*>(base);
            s_row_elem[r] = (unsigned char)elem;
            ++r;
        };
        auto close_group = [&](int first) {    // at most kGroupMax rows (grad_hess_tma_ok)
            s_gstart[ng] = (unsigned short)first;
            s_gsize[ng++] = (unsigned char)(r - first);
        };
        for (int k = 0; k < K; ++k) add_row(y + k * N, 4);
        if (b1p) add_row(b1p, 4);
        close_group(0);
        for (int c = 0; c < P.C; ++c) {
            const int first = r;
            if (b1m) add_row(b1m + c * N, 4);
            for (int e = 0; e < P.n_echoes[c]; ++e)
                add_row(x + (long long)(P.echo0[c] + e) * N, (int)sizeof(XT));
            close_group(first);
        }
        s_ngroups = ng;
    }
    __syncthreads();
    const int ng = s_ngroups;
    const int rows = s_gstart[ng - 1] + s_gsize[ng - 1];   // rows per chunk

    Acc nll_acc;
    unsigned gq_issued = 0;      // groups the producer issued
    if (warp == kGhWarps) {
        if (lane == 0 && !withhold) {
            unsigned q = 0, gq = 0, freed = 0;   // rows and groups issued, groups known released
            for (long long ch = vg.bx; ch < nchunks && !s_fail; ch += vg.gx) {
                const long long v0 = ch * kChunk;
                const uint32_t cnt = (uint32_t)min((long long)kChunk, N - v0);
                for (int gi = 0; gi < ng && !s_fail; ++gi) {
                    const int r = s_gsize[gi], r0 = s_gstart[gi];
                    // Before the copies: the group that last used this
                    // barrier, and every group holding a slot these rows
                    // take over (rows q - kSlots ... q + r - 1 - kSlots),
                    // must have been released.
                    while (freed < gq) {
                        const unsigned fstart = (freed / ng) * rows + s_gstart[freed % ng];
                        if (freed + kGroupBars > gq && fstart + kSlots >= q + r) break;
                        if (!mbar_wait_nap(smem_u32(&empty[freed % kGroupBars]), (freed / kGroupBars) & 1u,
                                           wait_cycles, 200)) {
                            s_fail = 1;
                            break;
                        }
                        ++freed;
                    }
                    // a compute warp that gave up released its group without
                    // the copies having landed: never put a second copy in
                    // flight to the same slot or barrier
                    if (s_fail) break;
                    uint32_t bytes = 0;
                    for (int k = 0; k < r; ++k) bytes += cnt * s_row_elem[r0 + k];
                    const uint32_t bar = smem_u32(&full[gq % kGroupBars]);
                    mbar_expect_tx(bar, bytes);
                    for (int k = 0; k < r; ++k) {
                        const int e = s_row_elem[r0 + k];
                        bulk_load(smem_u32(smem + ((q + k) % kSlots) * kSlotBytes),
                                  s_row_base[r0 + k] + v0 * e, cnt * e, bar);
                    }
                    q += r;
                    gq_issued = ++gq;
                }
            }
        }
    } else {
        const int t = tid;                      // compute thread 0 .. 223
        unsigned q = 0, gq = 0;                 // next row, next group
        bool bad = false;                       // a wait of this thread gave up
        // Group boundaries sit at fixed points of the code (the maps with
        // B1+, then one group per contrast): the first row waits for the
        // group's copies, the warp releases it after the last.  Rows are read
        // without branches: a thread past the end of the volume, or one whose
        // wait gave up, reads stale values and stores nothing.
        auto begin_group = [&]() {
            const uint32_t bar = smem_u32(&full[gq % kGroupBars]), par = (gq / kGroupBars) & 1u;
            bad = bad || s_fail || !(mbar_try_wait(bar, par) || mbar_wait_nap(bar, par, wait_cycles, 32));
            if (bad) s_fail = 1;
        };
        auto end_group = [&]() {
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&empty[gq % kGroupBars]));
            ++gq;
        };
        auto take = [&](auto tag, float (&o)[2]) {
            using E = decltype(tag);
            slot_pair(reinterpret_cast<const E*>(smem + (q % kSlots) * kSlotBytes) + 2 * t, o);
            ++q;
        };
        for (long long ch = vg.bx; ch < nchunks; ch += vg.gx) {
            const long long v0 = ch * kChunk;
            const long long n = v0 + 2 * t;
            const bool valid = n < N;           // N is a multiple of 8: pairs are whole
            float a[2], r1[2], r2[2], dl[2], m[2], bp[2] = {1.0f, 1.0f};
            begin_group();
            {
                float yv[K][2];
#pragma unroll
                for (int k = 0; k < K; ++k) take(float(), yv[k]);
                if (b1p) take(float(), bp);
                end_group();
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    float yk[4];
#pragma unroll
                    for (int k = 0; k < K; ++k) yk[k] = yv[k][v];
                    map_params_v(yk, K, a[v], r1[v], r2[v], dl[v], m[v]);
                }
            }
            float2 G[K], H[T], nll2 = make_float2(0.f, 0.f);   // x: first voxel, y: second
            Relax R[2];
#pragma unroll
            for (int k = 0; k < K; ++k) G[k] = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < T; ++k) H[k] = make_float2(0.f, 0.f);
#pragma unroll
            for (int v = 0; v < 2; ++v) R[v] = Relax{0.f, 0.f, 0.f};
            // Contrasts at contrast 0's flip angle reuse its flip factors, and
            // contrasts with the previous one's echo times its two echo
            // exponentials: the same values the unstaged pass recomputes.
            Flip f0[2];
            float2 e0 = make_float2(0.f, 0.f), rho = make_float2(0.f, 0.f);
            for (int c = 0; c < P.C; ++c) {
                begin_group();
                float bm[2] = {1.0f, 1.0f};
                if (b1m) take(float(), bm);
                ContrastTerms tc[2];
                const bool same_flip = (P.flip_as_c0 >> c) & 1u;
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    if (!P.same_tr[c]) R[v] = relax(P.tr[c], r1[v]);
                    const Flip f = same_flip ? f0[v] : flip(P.alpha[c] * bp[v]);
                    if (c == 0) f0[v] = f;
                    tc[v] = contrast_terms_f(P, c, a[v], R[v], dl[v], m[v], f, bm[v]);
                }
                // the echo loop of accumulate_contrast_v, echoes from the slots
                EchoSums2<PRE> es;
                const int i0 = P.echo0[c];
                const int ne = P.n_echoes[c];
                const float te0 = -P.te[i0];
                float2 q2 = make_float2(te0 * r2[0], te0 * r2[1]);
                float xv[2];
                if (P.te_uniform[c] != 0) {
                    const float dte = -P.dte[c];
                    const float2 dq = make_float2(dte * r2[0], dte * r2[1]);
                    if (!((P.echoes_as_prev >> c) & 1u)) {
                        e0 = make_float2(expf(q2.x), expf(q2.y));
                        rho = make_float2(expf(dq.x), expf(dq.y));
                    }
                    float2 sg = make_float2(tc[0].s0 * e0.x, tc[1].s0 * e0.y);
#pragma unroll 4
                    for (int e = 0; e < ne; ++e) {
                        take(XT(), xv);
                        es.add(sg, q2, make_float2(xv[0], xv[1]));
                        q2 = __fadd2_rn(q2, dq);
                        sg = __fmul2_rn(sg, rho);
                    }
                } else {
                    float2 sg = make_float2(tc[0].s0 * expf(q2.x), tc[1].s0 * expf(q2.y));
                    take(XT(), xv);
                    es.add(sg, q2, make_float2(xv[0], xv[1]));
#pragma unroll 4
                    for (int e = 1; e < ne; ++e) {
                        take(XT(), xv);
                        const float te = -P.te[i0 + e];
                        q2 = make_float2(te * r2[0], te * r2[1]);
                        sg = make_float2(tc[0].s0 * expf(q2.x), tc[1].s0 * expf(q2.y));
                        es.add(sg, q2, make_float2(xv[0], xv[1]));
                    }
                }
                end_group();
                finish_contrast2<K, PRE>(P, c, tc[0], tc[1], es, G, H, nll2);
            }
            if (valid && !bad) {
#pragma unroll
                for (int k = 0; k < K; ++k) *reinterpret_cast<float2*>(g + k * N + n) = G[k];
#pragma unroll
                for (int k = 0; k < T; ++k) *reinterpret_cast<float2*>(h + k * N + n) = H[k];
                nll_acc.add(nll2.x);
                nll_acc.add(nll2.y);
            }
        }
    }
    __syncthreads();
    if (s_fail) {
        // drain: no copy may still be writing this block's shared memory (the
        // last use of each group barrier; earlier groups were read, so their
        // copies completed, before their slots or barrier could be reused)
        if (warp == kGhWarps && lane == 0) {
            for (unsigned gq = gq_issued > kGroupBars ? gq_issued - kGroupBars : 0; gq < gq_issued; ++gq)
                mbar_wait(smem_u32(&full[gq % kGroupBars]), (gq / kGroupBars) & 1u, wait_cycles);
            if (status) atomicOr(status, kStatusTimeout);
        }
        __syncthreads();
    }
    Acc v[1] = {nll_acc};
    double out[1];
    if (grid_reduce<1>(v, red, out, vg) && tid == 0) *nll = out[0];
}

template <int K, int PRE, typename XT>
__global__ void __launch_bounds__(kGhThreads, 2)
    k_grad_hess_tma(DevProblem P, const XT* __restrict__ x, const float* __restrict__ y,
                    const float* __restrict__ b1p, const float* __restrict__ b1m,
                    float* __restrict__ g, float* __restrict__ h, double* nll, Reduce red,
                    unsigned* status, long long wait_cycles, int withhold)
{
    grad_hess_tma_body<K, PRE, XT>(P, x, y, b1p, b1m, g, h, nll, red, status, wait_cycles, withhold,
                                   hw_grid());
}

// Several subjects in one launch (batch.cuh): blocks [start[s], start[s + 1])
// run subject s's chunks.
template <int K, int PRE, typename XT>
__global__ void __launch_bounds__(kGhThreads, 2)
    k_grad_hess_tma_batch(const __grid_constant__ Batch<GradArgs> b, long long wait_cycles, int withhold)
{
    const int s = batch_subject(b.start, b.n);
    const GradArgs& a = b.a[s];
    grad_hess_tma_body<K, PRE, XT>(a.P, static_cast<const XT*>(a.x), a.y, a.b1p, a.b1m, a.g, a.h, a.nll,
                                   a.red, a.status, wait_cycles, withhold,
                                   batch_grid(b.start[s], b.start[s + 1] - b.start[s], 1, 1));
}

// Whether the staged pass applies: every row copy must start on a 16-byte
// boundary and move a multiple of 16 bytes, so N is a multiple of 8 and the
// arrays 16-byte aligned; and every group (a contrast's B1- and echoes) must
// fit half the ring.
bool grad_hess_tma_ok(const DevProblem& P, const void* x, const float* y, const float* b1p,
                      const float* b1m, const float* g, const float* h)
{
    auto al = [](const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; };
    if (!(P.N > 0 && P.N % 8 == 0 && al(x) && al(y) && al(b1p) && al(b1m) && al(g) && al(h)))
        return false;
    for (int c = 0; c < P.C; ++c)
        if (P.n_echoes[c] + (b1m ? 1 : 0) > kGroupMax) return false;
    return true;
}

static int sm_count()
{
    int sms = kNumSm, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = kNumSm;
    }
    return sms;
}

template <int K, int PRE, typename XT>
static cudaError_t launch_tma_k(const DevProblem& P, const void* x, const float* y, const float* b1p,
                                const float* b1m, float* g, float* h, double* nll, Reduce red,
                                unsigned* status, cudaStream_t st)
{
    auto* f = k_grad_hess_tma<K, PRE, XT>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kGhSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const long long chunks = (P.N + kChunk - 1) / kChunk;
    const int grid = (int)std::min<long long>(chunks, 2LL * sm_count());
    f<<<grid, kGhThreads, kGhSmem, st>>>(P, static_cast<const XT*>(x), y, b1p, b1m, g, h, nll, red,
                                         status, copy_wait_cycles(), copy_withhold());
    return cudaGetLastError();
}

template <int K, int PRE>
static cudaError_t launch_tma_dtype(const DevProblem& P, int echo_dtype, const void* x, const float* y,
                                    const float* b1p, const float* b1m, float* g, float* h,
                                    double* nll, Reduce red, unsigned* status, cudaStream_t st)
{
    if (echo_dtype == 1)
        return launch_tma_k<K, PRE, __nv_bfloat16>(P, x, y, b1p, b1m, g, h, nll, red, status, st);
    return launch_tma_k<K, PRE, float>(P, x, y, b1p, b1m, g, h, nll, red, status, st);
}

template <int K>
static cudaError_t launch_tma_pre(const DevProblem& P, int echo_dtype, const void* x, const float* y,
                                  const float* b1p, const float* b1m, float* g, float* h, double* nll,
                                  Reduce red, unsigned* status, cudaStream_t st)
{
    switch (P.precond) {
    case 0: return launch_tma_dtype<K, 0>(P, echo_dtype, x, y, b1p, b1m, g, h, nll, red, status, st);
    case 1: return launch_tma_dtype<K, 1>(P, echo_dtype, x, y, b1p, b1m, g, h, nll, red, status, st);
    default: return launch_tma_dtype<K, 2>(P, echo_dtype, x, y, b1p, b1m, g, h, nll, red, status, st);
    }
}

template <int K, int PRE, typename XT>
static cudaError_t launch_tma_batch_k(Batch<GradArgs>& b, cudaStream_t st)
{
    auto* f = k_grad_hess_tma_batch<K, PRE, XT>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kGhSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    f<<<b.start[b.n], kGhThreads, kGhSmem, st>>>(b, copy_wait_cycles(), copy_withhold());
    return cudaGetLastError();
}

template <int K, int PRE>
static cudaError_t launch_tma_batch_pre(int echo_dtype, Batch<GradArgs>& b, cudaStream_t st)
{
    if (echo_dtype == 1) return launch_tma_batch_k<K, PRE, __nv_bfloat16>(b, st);
    return launch_tma_batch_k<K, PRE, float>(b, st);
}

bool launch_grad_hess_tma_batch(int K, int precond, int echo_dtype, const GradArgs* a, int n,
                                cudaStream_t st, cudaError_t* err)
{
    long long total = 0;
    for (int s = 0; s < n; ++s) {
        if (!grad_hess_tma_ok(a[s].P, a[s].x, a[s].y, a[s].b1p, a[s].b1m, a[s].g, a[s].h)) return false;
        total += (a[s].P.N + kChunk - 1) / kChunk;
    }
    // one wave of two blocks per SM, shared in proportion to the chunks
    const long long wave = 2LL * sm_count();
    unsigned blocks[kBatchMax];
    for (int s = 0; s < n; ++s) {
        const long long c = (a[s].P.N + kChunk - 1) / kChunk;
        long long bs = (long long)std::llround((double)wave * (double)c / (double)total);
        blocks[s] = (unsigned)std::max(1LL, std::min(bs, c));
    }
    static thread_local Batch<GradArgs> b;
    fill_batch(b, a, blocks, n);
    switch (K * 10 + precond) {
    case 40: *err = launch_tma_batch_pre<4, 0>(echo_dtype, b, st); break;
    case 41: *err = launch_tma_batch_pre<4, 1>(echo_dtype, b, st); break;
    case 42: *err = launch_tma_batch_pre<4, 2>(echo_dtype, b, st); break;
    case 30: *err = launch_tma_batch_pre<3, 0>(echo_dtype, b, st); break;
    case 31: *err = launch_tma_batch_pre<3, 1>(echo_dtype, b, st); break;
    default: *err = launch_tma_batch_pre<3, 2>(echo_dtype, b, st); break;
    }
    return true;
}

template <int K, int PRE>
static cudaError_t prime_voxel_k()
{
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kGhSmem);
    };
    set(reinterpret_cast<const void*>(k_grad_hess_tma<K, PRE, float>));
    set(reinterpret_cast<const void*>(k_grad_hess_tma<K, PRE, __nv_bfloat16>));
    set(reinterpret_cast<const void*>(k_grad_hess_tma_batch<K, PRE, float>));
    set(reinterpret_cast<const void*>(k_grad_hess_tma_batch<K, PRE, __nv_bfloat16>));
    return e;
}

cudaError_t prime_voxel_kernels()
{
    cudaError_t e = prime_voxel_k<4, 0>();
    if (!e) e = prime_voxel_k<4, 1>();
    if (!e) e = prime_voxel_k<4, 2>();
    if (!e) e = prime_voxel_k<3, 0>();
    if (!e) e = prime_voxel_k<3, 1>();
    if (!e) e = prime_voxel_k<3, 2>();
    return e;
}

cudaError_t launch_grad_hess_tma(const DevProblem& P, int echo_dtype, const void* x, const float* y,
                                 const float* b1p, const float* b1m, float* g, float* h, double* nll,
                                 Reduce red, unsigned* status, cudaStream_t st)
{
    if (P.K == 4) return launch_tma_pre<4>(P, echo_dtype, x, y, b1p, b1m, g, h, nll, red, status, st);
    return launch_tma_pre<3>(P, echo_dtype, x, y, b1p, b1m, g, h, nll, red, status, st);
}

}  // namespace mpm
