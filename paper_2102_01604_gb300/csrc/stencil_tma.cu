// stencil_tma.cu -- one PCG iteration of the Newton system (Eq. 42) with
// TMA plane staging (sm_103a).  The per-voxel arithmetic is pcg_step.cuh's,
// shared with the plain kernel k_pcg_step (stencil_kernels.cu).
//
// Iteration j reads z_{j-1}, v_{j-1} and p_{j-1} (with a one-voxel halo), the
// JTV weights and H, and writes z_j, p_j and v_j once:
//   z_j = z_{j-1} - alpha_{j-1} v_{j-1},  p_j = z_j + beta_{j-1} p_{j-1}
//   q_j = (H + L) p_j,  v_j = M^-1 q_j,  and the sums for alpha_j and beta_j.
// A block owns a TX x TY tile and marches up a run of z planes.  Per plane
// one thread issues bulk tensor copies into a ring of "raw" stages:
//   z, v, p   (TX+2) x (TY+2) voxels of 4 floats at (x0 - 1, y0 - 1, z)
//   w         (TX+8) x (TY+2) floats at (x0 - 4, y0 - 1, z)
//   x, p_j-2  TX x TY voxels of 4 floats at (x0, y0, z) (even j >= 2, x fold)
// and H (TX x TY x T floats, planar) into a second ring.  The solve's own
// vectors hold 4 floats per voxel, so their boxes start 16-byte aligned at
// any x; the planar w box starts at a multiple of 4 floats.  Boxes that leave
// the volume are zero-filled by the copy engine and masked by zero stencil
// coefficients.
//
// The compute warps (one voxel per thread) take each plane in two phases:
//   A  form z_j and p_j of the plane's points (the tile and its x / y halo,
//      recomputed from the staged z, v, p) into a shared "formed" plane (a
//      ring of three), write z_j and p_j of the tile and fold x; the raw
//      stage is then released;
//   B  one plane behind A: q = (H + L) p_j from the formed plane (x / y
//      neighbours) and the thread's own column (z neighbours, kept in
//      registers), v = M^-1 q, r = M z_j, the voxel's terms of the sums.
// One named barrier among the compute warps per plane separates A's writes
// of a formed plane from B's reads of it; with three formed planes in the
// ring, A never overwrites a plane B may still read.  A producer warp keeps
// both rings full; a stage is refilled once all compute warps have released
// it.  Each thread sums its voxels' terms in float32 over one item
// (at most one z range of its column) and adds that partial to compensated
// accumulators, which the block and the grid reduce in float64.
//
// Every mbarrier wait is bounded: on timeout the block records
// kStatusTimeout, stops computing (its warps still pass the same named
// barriers, so none waits forever), drains its outstanding copies (bounded
// again) and still takes part in the grid reduction.
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include "mpm_internal.cuh"
#include "pcg_step.cuh"
#include "tma_common.cuh"

namespace mpm {

constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz

// Test hooks (mpm_test_copy_timeout): the producers of the staged kernels
// issue no copies, and the bound of every wait, in clock cycles.
static std::atomic<int> g_withhold{0};
static std::atomic<long long> g_wait_cycles{kWaitCycles};

void set_copy_test(int withhold, long long wait_cycles)
{
    g_withhold.store(withhold ? 1 : 0);
    g_wait_cycles.store(wait_cycles > 0 ? wait_cycles : kWaitCycles);
}

int copy_withhold() { return g_withhold.load(std::memory_order_relaxed); }
long long copy_wait_cycles() { return g_wait_cycles.load(std::memory_order_relaxed); }

// Per tile shape: one compute thread per voxel plus a producer warp.  256-
// voxel tiles run two blocks per SM with two raw stages in the x-fold
// iterations (whose stages also hold the x and p_{j-2} tiles) and three in
// the others; 512-voxel tiles one block per SM with three and four.
template <int K, int TX, int TY, bool FOLD = true>
struct StepLayout {
    static constexpr int VOX = TX * TY;                 // voxels per tile = compute threads
    static constexpr int WARPS = VOX / 32;              // compute warps
    static constexpr int THREADS = VOX + 32;            // plus the producer warp
    static constexpr int MINB = VOX >= 512 ? 1 : 2;     // resident blocks per SM aimed for
    static constexpr int RS = (VOX >= 512 ? 3 : 2) + (FOLD ? 0 : 1);   // raw (z, v, p, w[, x, p_{j-2}]) stages
    static constexpr int HS = FOLD ? 2 : 3;             // H stages
    static constexpr int T = K * (K + 1) / 2;
    static constexpr int BX = TX + 2, BY = TY + 2;      // z / v / p box and formed plane (x from x0 - 1)
    static constexpr int WX = TX + 8;                   // w box (x from x0 - 4, 16-byte aligned)
    static constexpr int NH = 2 * (TX + TY);            // halo points of a formed plane
    static constexpr int a128(int b) { return (b + 127) / 128 * 128; }
    static constexpr int BOX_BYTES = BX * BY * 16, W_BYTES = WX * BY * 4;
    static constexpr int TILE_BYTES = TX * TY * 16, H_BYTES = T * TX * TY * 4;
    static constexpr int Z_OFF = 0;
    static constexpr int V_OFF = a128(BOX_BYTES);
    static constexpr int P_OFF = V_OFF + a128(BOX_BYTES);
    static constexpr int W_OFF = P_OFF + a128(BOX_BYTES);
    static constexpr int X_OFF = W_OFF + a128(W_BYTES);
    static constexpr int P2_OFF = X_OFF + a128(TILE_BYTES);
    static constexpr int RAW = FOLD ? P2_OFF + a128(TILE_BYTES) : X_OFF;
    static constexpr int H_STAGE = a128(H_BYTES);
    static constexpr int SLOT = a128(BOX_BYTES);
    static constexpr int H_BASE = RS * RAW;
    static constexpr int S_BASE = H_BASE + HS * H_STAGE;
    static constexpr int SMEM = S_BASE + 3 * SLOT + 128;   // + alignment slack
    static_assert(VOX % 32 == 0, "whole compute warps");
    static_assert(NH <= VOX, "one halo point per thread at most");
    static_assert(SMEM <= 227 * 1024, "shared memory of one block");
    static_assert(4 * BX <= 256 && 4 * TX <= 256, "TMA box rows of at most 256 elements");
};

// Dynamic shared memory a step kernel of this tile shape asks for: the larger
// of the two layouts, so that every mode's launch fits the same opt-in and the
// occupancy query holds for both.
template <int K, int TX, int TY>
constexpr int step_smem_max()
{
    return StepLayout<K, TX, TY, true>::SMEM > StepLayout<K, TX, TY, false>::SMEM
               ? StepLayout<K, TX, TY, true>::SMEM
               : StepLayout<K, TX, TY, false>::SMEM;
}

// Barrier 1 among the compute warps (the producer warp never joins it).
template <int NTHREADS>
__device__ __forceinline__ void compute_warps_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(NTHREADS) : "memory");
}

// Work split: the launch is one wave of resident blocks.  The volume is cut
// into items -- one tile column over one of `nchunk` z ranges -- numbered
// i = chunk * tiles + tile, and block b takes items b, b + G, b + 2G, ...
// (G = gridDim.x), so the blocks running at one time cover neighbouring
// tiles of the same z ranges (their DRAM rows and halos are shared).  An item
// over planes [za, zb) loads planes za - 1 .. zb (those inside the volume);
// the planes outside [za, zb) only supply the z neighbours of its own column.
// The rings and their phases run on from one item to the next.
template <int K, int TX, int TY, int MODE>
__device__ __forceinline__ void step_body(
    const DevProblem& P, int nchunk, int j, int want_rr, const CUtensorMap* tz, const CUtensorMap* tv,
    const CUtensorMap* tp, const CUtensorMap* tw, const CUtensorMap* th, const CUtensorMap* txm,
    const CUtensorMap* tp2, float4* __restrict__ zout, float4* __restrict__ vout,
    float4* __restrict__ pout, float4* __restrict__ xacc, WsHeader* hdr, double* resid, Reduce red,
    long long wait_cycles, int withhold, const VGrid& vg)
{
    using L = StepLayout<K, TX, TY, (MODE >= kModeFold)>;
    constexpr int T = L::T;
    constexpr int kStepRaw = L::RS, kStepH = L::HS, kStepWarps = L::WARPS;
    constexpr bool first = MODE == kModeFirst, fold = MODE >= kModeFold, readx = MODE == kModeFoldX;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t raw_full[kStepRaw], raw_empty[kStepRaw];
    __shared__ __align__(8) uint64_t h_full[kStepH], h_empty[kStepH];
    __shared__ int s_done;
    __shared__ float s_alpha, s_alpha_prev, s_beta;
    __shared__ volatile int s_fail;
    unsigned char* smem =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const bool producer = warp == kStepWarps;
    const int tx = tid % TX, ty = tid / TX;              // meaningful for compute threads
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int gx = (nx + TX - 1) / TX;
    const int tiles = gx * ((ny + TY - 1) / TY);
    const int items = tiles * nchunk;

    if (tid == 0) {
        s_done = hdr->sc.done;
        s_alpha = (float)hdr->sc.alpha;
        s_alpha_prev = (float)hdr->sc.alpha_prev;
        s_beta = (float)hdr->sc.beta;
        s_fail = 0;
        for (int s = 0; s < kStepRaw; ++s) {
            mbar_init(smem_u32(&raw_full[s]), 1);
            mbar_init(smem_u32(&raw_empty[s]), kStepWarps);
        }
        for (int s = 0; s < kStepH; ++s) {
            mbar_init(smem_u32(&h_full[s]), 1);
            mbar_init(smem_u32(&h_empty[s]), kStepWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (s_done) return;                                   // the same in every block
    if (fold && tid == 0 && vg.bx == 0) hdr->sc.xcount = j;
    const float alpha = s_alpha, alpha_prev = s_alpha_prev, beta = s_beta;

    // Counters: c over the raw planes this block loads, e over its H planes
    // (one per plane it computes), both in order -> ring stage and phase.
    auto r_stage = [](int c) { return (int)((unsigned)c % (unsigned)kStepRaw); };
    auto r_phase = [](int c) { return (uint32_t)(((unsigned)c / (unsigned)kStepRaw) & 1u); };
    auto h_stage = [](int e) { return (int)((unsigned)e % (unsigned)kStepH); };
    auto h_phase = [](int e) { return (uint32_t)(((unsigned)e / (unsigned)kStepH) & 1u); };
    auto formed = [&](int c) {
        return reinterpret_cast<float4*>(smem + L::S_BASE + ((unsigned)c % 3u) * L::SLOT);
    };

    Acc acc[kStepSums];
    int raw_issued = -1, h_issued = -1;   // last counters issued (producer lane 0)
    if (producer) {
        if (lane == 0 && !withhold) {
            int cb = 0, eb = 0;           // counters of the item's first planes
            for (int i = (int)vg.bx; i < items && !s_fail; i += (int)vg.gx) {
                const int t = i % tiles, ch = i / tiles;
                const int za = (int)((long long)ch * nz / nchunk), zb = (int)((long long)(ch + 1) * nz / nchunk);
                const int x0 = (t % gx) * TX, y0 = (t / gx) * TY;
                const int ja = max(za - 1, 0), jb = min(zb, nz - 1);
                for (int jj = ja; jj <= jb && !s_fail; ++jj) {
                    const int c = cb + (jj - ja);
                    const int s = r_stage(c);
                    if (c >= kStepRaw &&
                        !mbar_wait(smem_u32(&raw_empty[s]), r_phase(c - kStepRaw), wait_cycles)) {
                        s_fail = 1;
                        break;
                    }
                    const bool inner = jj >= za && jj < zb;
                    unsigned char* st = smem + s * L::RAW;
                    const uint32_t bar = smem_u32(&raw_full[s]);
                    uint32_t bytes = L::BOX_BYTES + L::W_BYTES;
                    if (!first) bytes += 2 * L::BOX_BYTES;
                    if (fold && inner) bytes += L::TILE_BYTES * (readx ? 2 : 1);
                    mbar_expect_tx(bar, bytes);
                    tma_load_3d(smem_u32(st + L::Z_OFF), tz, 4 * (x0 - 1), y0 - 1, jj, bar);
                    if (!first) {
                        tma_load_3d(smem_u32(st + L::V_OFF), tv, 4 * (x0 - 1), y0 - 1, jj, bar);
                        tma_load_3d(smem_u32(st + L::P_OFF), tp, 4 * (x0 - 1), y0 - 1, jj, bar);
                    }
                    tma_load_3d(smem_u32(st + L::W_OFF), tw, x0 - 4, y0 - 1, jj, bar);
                    if (fold && inner) {
                        tma_load_3d(smem_u32(st + L::P2_OFF), tp2, 4 * x0, y0, jj, bar);
                        if (readx) tma_load_3d(smem_u32(st + L::X_OFF), txm, 4 * x0, y0, jj, bar);
                    }
                    raw_issued = c;
                    if (!inner) continue;
                    const int e = eb + (jj - za);
                    const int sh = h_stage(e);
                    if (e >= kStepH &&
                        !mbar_wait(smem_u32(&h_empty[sh]), h_phase(e - kStepH), wait_cycles)) {
                        s_fail = 1;
                        break;
                    }
                    const uint32_t hbar = smem_u32(&h_full[sh]);
                    mbar_expect_tx(hbar, L::H_BYTES);
                    tma_load_4d(smem_u32(smem + L::H_BASE + sh * L::H_STAGE), th, x0, y0, jj, 0, hbar);
                    h_issued = e;
                }
                cb += jb - ja + 1;
                eb += zb - za;
            }
        }
    } else {
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        int cb = 0, eb = 0;
        for (int i = (int)vg.bx; i < items; i += (int)vg.gx) {
            const int t = i % tiles, ch = i / tiles;
            const int za = (int)((long long)ch * nz / nchunk), zb = (int)((long long)(ch + 1) * nz / nchunk);
            const int x = (t % gx) * TX + tx, y = (t / gx) * TY + ty;
            const int ja = max(za - 1, 0), jb = min(zb, nz - 1);
            const bool inside = x < nx && y < ny;
            const bool okxm = x > 0, okxp = x + 1 < nx, okym = y > 0, okyp = y + 1 < ny;
            const int bc = (ty + 1) * L::BX + tx + 1;      // own point in a z / v / p box and formed plane
            const int wcc = (ty + 1) * L::WX + tx + 4;     // own point in a w box
            const int tc = ty * TX + tx;                   // own point in a tile box
            // own column: p_j of planes z - 1, z, z + 1, z_j of z and z + 1,
            // the weights of z - 1, z, z + 1 and the x / y coefficients of z, z + 1
            float pm[K], pc[K], pn[K], zc[K], zn[K], cxy[4], cxyn[4];
            float wm = 0.f, wc = 0.f, wn = 0.f;
#pragma unroll
            for (int a = 0; a < K; ++a) pm[a] = pc[a] = pn[a] = zc[a] = zn[a] = 0.f;
#pragma unroll
            for (int m = 0; m < 4; ++m) cxy[m] = cxyn[m] = 0.f;
            float part[kStepSums] = {};
            const long long col = (long long)x + (long long)nx * y;
            const long long sxy = (long long)nx * ny;

            // Phase B for plane z (counter cz of its formed plane, H counter e):
            // `up` holds p_j of plane z + 1 (or of z itself at the top face).
            auto phase_b = [&](int z, int cz, int e, const float (&up)[K], float wup) {
                const bool ok = !s_fail && mbar_wait(smem_u32(&h_full[h_stage(e)]), h_phase(e), wait_cycles);
                if (!ok) s_fail = 1;
                if (ok && inside) {
                    const float* hb = reinterpret_cast<const float*>(smem + L::H_BASE + h_stage(e) * L::H_STAGE);
                    float hv[T];
#pragma unroll
                    for (int m = 0; m < T; ++m) hv[m] = hb[m * TX * TY + tc];
                    const float4* fp = formed(cz);
                    float nb[4][K];
                    unpack4<K>(fp[bc - 1], nb[0]);
                    unpack4<K>(fp[bc + 1], nb[1]);
                    unpack4<K>(fp[bc - L::BX], nb[2]);
                    unpack4<K>(fp[bc + L::BX], nb[3]);
                    const float c6[6] = {cxy[0], cxy[1], cxy[2], cxy[3],
                                         z > 0 ? (wc + wm) * P.ihz2 : 0.f,
                                         z + 1 < nz ? (wc + wup) * P.ihz2 : 0.f};
                    auto nbf = [&](int m, int a) -> float {
                        return m < 4 ? nb[m][a] : (m == 4 ? pm[a] : up[a]);
                    };
                    float v[K], sums[kStepSums];
                    step_voxel<K>(P, c6, zc, pc, nbf, hv, want_rr, v, sums);
                    vout[col + sxy * z] = pack4<K>(v);
#pragma unroll
                    for (int s = 0; s < kStepSums; ++s) part[s] += sums[s];
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&h_empty[h_stage(e)]));
            };

            for (int jj = ja; jj <= jb; ++jj) {
                const int c = cb + (jj - ja);
                const bool inner = jj >= za && jj < zb;
                const bool ok = !s_fail && mbar_wait(smem_u32(&raw_full[r_stage(c)]), r_phase(c), wait_cycles);
                if (!ok) s_fail = 1;
                if (ok) {
                    // Phase A: z_j and p_j of this plane
                    const unsigned char* st = smem + r_stage(c) * L::RAW;
                    const float4* bz = reinterpret_cast<const float4*>(st + L::Z_OFF);
                    const float4* bv = reinterpret_cast<const float4*>(st + L::V_OFF);
                    const float4* bp = reinterpret_cast<const float4*>(st + L::P_OFF);
                    const float* bw = reinterpret_cast<const float*>(st + L::W_OFF);
                    const float4 p4 = first ? zero4 : bp[bc];
                    step_point<K, first>(alpha, beta, bz[bc], first ? zero4 : bv[bc], p4, zn, pn);
                    wn = bw[wcc];
                    cxyn[0] = okxm ? (wn + bw[wcc - 1]) * P.ihx2 : 0.f;
                    cxyn[1] = okxp ? (wn + bw[wcc + 1]) * P.ihx2 : 0.f;
                    cxyn[2] = okym ? (wn + bw[wcc - L::WX]) * P.ihy2 : 0.f;
                    cxyn[3] = okyp ? (wn + bw[wcc + L::WX]) * P.ihy2 : 0.f;
                    if (inner) {
                        float4* fp = formed(c);
                        fp[bc] = pack4<K>(pn);
                        if (tid < L::NH) {
                            // halo point: y - 1 row, y + TY row, x - 1 column, x + TX column
                            int hb;
                            if (tid < TX) hb = tid + 1;
                            else if (tid < 2 * TX) hb = (TY + 1) * L::BX + tid - TX + 1;
                            else if (tid < 2 * TX + TY) hb = (tid - 2 * TX + 1) * L::BX;
                            else hb = (tid - 2 * TX - TY + 1) * L::BX + TX + 1;
                            float hzj[K], hpj[K];
                            step_point<K, first>(alpha, beta, bz[hb], first ? zero4 : bv[hb],
                                                 first ? zero4 : bp[hb], hzj, hpj);
                            fp[hb] = pack4<K>(hpj);
                        }
                        if (inside) {
                            const long long n = col + sxy * jj;
                            if (!first) zout[n] = pack4<K>(zn);
                            pout[n] = pack4<K>(pn);
                            if (fold) {
                                const float4* bx = reinterpret_cast<const float4*>(st + L::X_OFF);
                                const float4* b2 = reinterpret_cast<const float4*>(st + L::P2_OFF);
                                xacc[n] = fold_x(readx ? bx[tc] : zero4, alpha_prev, b2[tc], alpha, p4);
                            }
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&raw_empty[r_stage(c)]));
                compute_warps_sync<L::VOX>();
                if (jj - 1 >= za) phase_b(jj - 1, c - 1, eb + (jj - 1 - za), pn, wn);
                // the plane above becomes current
#pragma unroll
                for (int a = 0; a < K; ++a) {
                    pm[a] = pc[a];
                    pc[a] = pn[a];
                    zc[a] = zn[a];
                }
#pragma unroll
                for (int m = 0; m < 4; ++m) cxy[m] = cxyn[m];
                wm = wc;
                wc = wn;
            }
            if (jb == zb - 1) {
                // the item reaches the top face: its last plane has no plane above
                phase_b(jb, cb + (jb - ja), eb + (jb - za), pc, wc);
            }
            cb += jb - ja + 1;
            eb += zb - za;
#pragma unroll
            for (int s = 0; s < kStepSums; ++s) {
                acc[s].add(part[s]);
                part[s] = 0.f;
            }
        }
    }
    __syncthreads();
    if (s_fail) {
        // drain: no copy may still be writing this block's shared memory
        if (producer && lane == 0) {
            // the last fill of each stage (earlier fills have completed before
            // their stage could be refilled)
            for (int c = max(0, raw_issued - kStepRaw + 1); c <= raw_issued; ++c)
                mbar_wait(smem_u32(&raw_full[r_stage(c)]), r_phase(c), wait_cycles);
            for (int e = max(0, h_issued - kStepH + 1); e <= h_issued; ++e)
                mbar_wait(smem_u32(&h_full[h_stage(e)]), h_phase(e), wait_cycles);
            atomicOr(&hdr->status, kStatusTimeout);
        }
        __syncthreads();
    }
    double out[kStepSums];
    if (grid_reduce<kStepSums>(acc, red, out, vg) && tid == 0) step_scalars(out, j, want_rr, hdr, resid);
}

template <int K, int TX, int TY, int MODE>
__global__ void __launch_bounds__(StepLayout<K, TX, TY>::THREADS, StepLayout<K, TX, TY>::MINB) k_pcg_step_tma(
    DevProblem P, int nchunk, int j, int want_rr, const __grid_constant__ CUtensorMap tz,
    const __grid_constant__ CUtensorMap tv, const __grid_constant__ CUtensorMap tp,
    const __grid_constant__ CUtensorMap tw, const __grid_constant__ CUtensorMap th,
    const __grid_constant__ CUtensorMap txm, const __grid_constant__ CUtensorMap tp2,
    float4* __restrict__ zout, float4* __restrict__ vout, float4* __restrict__ pout,
    float4* __restrict__ xacc, WsHeader* hdr, double* resid, Reduce red, long long wait_cycles,
    int withhold)
{
    step_body<K, TX, TY, MODE>(P, nchunk, j, want_rr, &tz, &tv, &tp, &tw, &th, &txm, &tp2, zout, vout,
                               pout, xacc, hdr, resid, red, wait_cycles, withhold, hw_grid());
}

// Several subjects in one launch (mpm_fit_batch with opts.graph = 2).
template <int K, int TX, int TY, int MODE>
__global__ void __launch_bounds__(StepLayout<K, TX, TY>::THREADS, StepLayout<K, TX, TY>::MINB)
    k_pcg_step_tma_batch(const __grid_constant__ Batch<StepArgs> b)
{
    const int s = batch_subject(b.start, b.n);
    const StepArgs& a = b.a[s];
    step_body<K, TX, TY, MODE>(a.P, a.nchunk, a.j, a.want_rr, &a.tz, &a.tv, &a.tp, &a.tw, &a.th, &a.tx,
                               &a.tp2, a.zout, a.vout, a.pout, a.xacc, a.hdr, a.resid, a.red,
                               a.wait_cycles, a.withhold, batch_grid(b.start[s], b.start[s + 1] - b.start[s], 1, 1));
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
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int tma_wave(const DevProblem& P, int tile);

// Tile shapes the TMA iteration is compiled for (x by y voxels).
static const int kTileShapes[][2] = {{16, 16}, {32, 8}, {32, 16}};

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

bool make_step_maps(const DevProblem& P, const float* h, const float* w, const SolveBufs& B, int tile,
                    StepMaps* out)
{
    if (tile < 0 || tile >= tma_tile_count()) return false;
    const int TX = kTileShapes[tile][0], TY = kTileShapes[tile][1];
    const int BX = TX + 2, BY = TY + 2, WX = TX + 8;
    // The planar maps need 16-byte row strides (nx a multiple of 4); boxes
    // are kept no larger than the volume; every base must be 16-byte aligned.
    if (P.nx % 4 != 0 || P.nx < WX || P.ny < BY) return false;
    uintptr_t any = reinterpret_cast<uintptr_t>(h) | reinterpret_cast<uintptr_t>(w) |
                    reinterpret_cast<uintptr_t>(B.x);
    for (float4* v : B.z) any |= reinterpret_cast<uintptr_t>(v);
    for (float4* v : B.v) any |= reinterpret_cast<uintptr_t>(v);
    for (float4* v : B.p) any |= reinterpret_cast<uintptr_t>(v);
    if (any % 16) return false;
    if (!encode_fn()) return false;
    const cuuint64_t nx = P.nx, ny = P.ny, nz = P.nz;
    // voxel-interleaved vectors: 4 nx floats per row
    const cuuint64_t da[3] = {4 * nx, ny, nz};
    const cuuint64_t sa[2] = {16 * nx, 16 * nx * ny};
    const cuuint32_t halo[3] = {(cuuint32_t)(4 * BX), (cuuint32_t)BY, 1};
    const cuuint32_t tilebox[3] = {(cuuint32_t)(4 * TX), (cuuint32_t)TY, 1};
    // planar arrays
    const cuuint64_t d3[3] = {nx, ny, nz};
    const cuuint64_t s3[2] = {4 * nx, 4 * nx * ny};
    const cuuint64_t dh[4] = {nx, ny, nz, (cuuint64_t)P.T};
    const cuuint64_t sh[3] = {4 * nx, 4 * nx * ny, 4 * (cuuint64_t)P.N};
    const cuuint32_t wbox[3] = {(cuuint32_t)WX, (cuuint32_t)BY, 1};
    const cuuint32_t hbox[4] = {(cuuint32_t)TX, (cuuint32_t)TY, 1, (cuuint32_t)P.T};
    auto f = [](const float4* v) { return reinterpret_cast<const float*>(v); };
    bool ok = encode(&out->w, w, 3, d3, s3, wbox) && encode(&out->h, h, 4, dh, sh, hbox) &&
              encode(&out->x, f(B.x), 3, da, sa, tilebox);
    for (int i = 0; i < 2 && ok; ++i)
        ok = encode(&out->z[i], f(B.z[i]), 3, da, sa, halo) && encode(&out->v[i], f(B.v[i]), 3, da, sa, halo);
    for (int i = 0; i < 3 && ok; ++i)
        ok = encode(&out->p[i], f(B.p[i]), 3, da, sa, halo) &&
             encode(&out->p2[i], f(B.p[i]), 3, da, sa, tilebox);
    out->B = B;
    out->tile = tile;
    return ok;
}

template <int K, int TX, int TY, int MODE>
static cudaError_t launch_step_m(const DevProblem& P, int nchunk, dim3 grid, const StepMaps& m, int j,
                                 int want_rr, WsHeader* hdr, double* resid, Reduce red, cudaStream_t st)
{
    using L = StepLayout<K, TX, TY, (MODE >= kModeFold)>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_pcg_step_tma<K, TX, TY, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             step_smem_max<K, TX, TY>());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int jm = j > 0 ? j - 1 : 0;
    k_pcg_step_tma<K, TX, TY, MODE><<<grid, dim3(L::THREADS, 1, 1), L::SMEM, st>>>(
        P, nchunk, j, want_rr, m.z[jm & 1], m.v[jm & 1], m.p[(j + 2) % 3], m.w, m.h, m.x,
        m.p2[(j + 1) % 3], m.B.z[j & 1], m.B.v[j & 1], m.B.p[j % 3], m.B.x, hdr, resid, red,
        g_wait_cycles.load(std::memory_order_relaxed), g_withhold.load(std::memory_order_relaxed));
    return cudaGetLastError();
}

template <int K, int TX, int TY>
static cudaError_t launch_step_k(const DevProblem& P, int nchunk, dim3 grid, const StepMaps& m, int j,
                                 int mode, int want_rr, WsHeader* hdr, double* resid, Reduce red,
                                 cudaStream_t st)
{
    switch (mode) {
    case kModeFirst: return launch_step_m<K, TX, TY, kModeFirst>(P, nchunk, grid, m, j, want_rr, hdr, resid, red, st);
    case kModeStep: return launch_step_m<K, TX, TY, kModeStep>(P, nchunk, grid, m, j, want_rr, hdr, resid, red, st);
    case kModeFold: return launch_step_m<K, TX, TY, kModeFold>(P, nchunk, grid, m, j, want_rr, hdr, resid, red, st);
    default: return launch_step_m<K, TX, TY, kModeFoldX>(P, nchunk, grid, m, j, want_rr, hdr, resid, red, st);
    }
}

StepArgs step_args(const DevProblem& P, const StepMaps& m, int nchunk, int j, int want_rr,
                   WsHeader* hdr, double* resid, Reduce red)
{
    StepArgs a;
    const int jm = j > 0 ? j - 1 : 0;
    a.tz = m.z[jm & 1];
    a.tv = m.v[jm & 1];
    a.tp = m.p[(j + 2) % 3];
    a.tw = m.w;
    a.th = m.h;
    a.tx = m.x;
    a.tp2 = m.p2[(j + 1) % 3];
    a.P = P;
    a.nchunk = nchunk;
    a.j = j;
    a.want_rr = want_rr;
    a.zout = m.B.z[j & 1];
    a.vout = m.B.v[j & 1];
    a.pout = m.B.p[j % 3];
    a.xacc = m.B.x;
    a.hdr = hdr;
    a.resid = resid;
    a.red = red;
    a.wait_cycles = g_wait_cycles.load(std::memory_order_relaxed);
    a.withhold = g_withhold.load(std::memory_order_relaxed);
    return a;
}

template <int K, int TX, int TY, int MODE>
static cudaError_t launch_step_batch_m(const Batch<StepArgs>& b, cudaStream_t st)
{
    using L = StepLayout<K, TX, TY, (MODE >= kModeFold)>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_pcg_step_tma_batch<K, TX, TY, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             step_smem_max<K, TX, TY>());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_pcg_step_tma_batch<K, TX, TY, MODE><<<b.start[b.n], dim3(L::THREADS, 1, 1), L::SMEM, st>>>(b);
    return cudaGetLastError();
}

template <int K, int TX, int TY>
static cudaError_t launch_step_batch_k(int mode, const Batch<StepArgs>& b, cudaStream_t st)
{
    switch (mode) {
    case kModeFirst: return launch_step_batch_m<K, TX, TY, kModeFirst>(b, st);
    case kModeStep: return launch_step_batch_m<K, TX, TY, kModeStep>(b, st);
    case kModeFold: return launch_step_batch_m<K, TX, TY, kModeFold>(b, st);
    default: return launch_step_batch_m<K, TX, TY, kModeFoldX>(b, st);
    }
}

cudaError_t launch_step_batch(int K, int tile, int mode, const StepArgs* a, const unsigned* blocks,
                              int n, cudaStream_t st)
{
    static thread_local Batch<StepArgs> b;   // 27 KB, kept off the stack
    fill_batch(b, a, blocks, n);
    LaunchScope ls(MPM_KERNEL_PCG_STEP, st);
    if (K == 4) {
        if (tile == 2) return launch_step_batch_k<4, 32, 16>(mode, b, st);
        if (tile == 1) return launch_step_batch_k<4, 32, 8>(mode, b, st);
        return launch_step_batch_k<4, 16, 16>(mode, b, st);
    }
    if (tile == 2) return launch_step_batch_k<3, 32, 16>(mode, b, st);
    if (tile == 1) return launch_step_batch_k<3, 32, 8>(mode, b, st);
    return launch_step_batch_k<3, 16, 16>(mode, b, st);
}

int tma_tiles_of(const DevProblem& P, int tile)
{
    const int TX = kTileShapes[tile][0], TY = kTileShapes[tile][1];
    return ((P.nx + TX - 1) / TX) * ((P.ny + TY - 1) / TY);
}

int tma_wave_blocks(const DevProblem& P, int tile) { return tma_wave(P, tile); }

template <int K, int TX, int TY>
static int resident_one()
{
    // the occupancy query needs the kernel's shared-memory opt-in first
    int nb = 0;
    if (cudaFuncSetAttribute(k_pcg_step_tma<K, TX, TY, kModeFoldX>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, step_smem_max<K, TX, TY>()) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pcg_step_tma<K, TX, TY, kModeFoldX>,
                                                      StepLayout<K, TX, TY>::THREADS,
                                                      step_smem_max<K, TX, TY>()) !=
            cudaSuccess) {
        cudaGetLastError();
        nb = 1;
    }
    return nb > 0 ? nb : 1;
}

// Resident blocks of the TMA iteration per SM for (K, tile) times the SM
// count of the current device, looked up once per device.
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
        nb = tile == 2 ? resident_one<4, 32, 16>() : tile == 1 ? resident_one<4, 32, 8>() : resident_one<4, 16, 16>();
    else
        nb = tile == 2 ? resident_one<3, 32, 16>() : tile == 1 ? resident_one<3, 32, 8>() : resident_one<3, 16, 16>();
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
    g.block = dim3(tile == 2 ? StepLayout<4, 32, 16>::THREADS : StepLayout<4, 16, 16>::THREADS, 1, 1);
    g.zc = best;
    return g;
}

template <int K, int TX, int TY>
static cudaError_t prime_one()
{
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     step_smem_max<K, TX, TY>());
    };
    set(reinterpret_cast<const void*>(k_pcg_step_tma<K, TX, TY, kModeFirst>));
    set(reinterpret_cast<const void*>(k_pcg_step_tma<K, TX, TY, kModeStep>));
    set(reinterpret_cast<const void*>(k_pcg_step_tma<K, TX, TY, kModeFold>));
    set(reinterpret_cast<const void*>(k_pcg_step_tma<K, TX, TY, kModeFoldX>));
    set(reinterpret_cast<const void*>(k_pcg_step_tma_batch<K, TX, TY, kModeFirst>));
    set(reinterpret_cast<const void*>(k_pcg_step_tma_batch<K, TX, TY, kModeStep>));
    set(reinterpret_cast<const void*>(k_pcg_step_tma_batch<K, TX, TY, kModeFold>));
    set(reinterpret_cast<const void*>(k_pcg_step_tma_batch<K, TX, TY, kModeFoldX>));
    return e;
}

cudaError_t prime_tma_kernels()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = prime_voxel_kernels();
    if (!e) e = prime_one<4, 16, 16>();
    if (!e) e = prime_one<4, 32, 8>();
    if (!e) e = prime_one<4, 32, 16>();
    if (!e) e = prime_one<3, 16, 16>();
    if (!e) e = prime_one<3, 32, 8>();
    if (!e) e = prime_one<3, 32, 16>();
    if (!e) done = true;
    return e;
}

cudaError_t launch_step_tma(const DevProblem& P, const StencilGrid& g, const StepMaps& m, int j,
                            int mode, int want_rr, WsHeader* hdr, double* resid, Reduce red,
                            cudaStream_t st)
{
    if (P.K == 4) {
        if (m.tile == 2) return launch_step_k<4, 32, 16>(P, g.zc, g.grid, m, j, mode, want_rr, hdr, resid, red, st);
        if (m.tile == 1) return launch_step_k<4, 32, 8>(P, g.zc, g.grid, m, j, mode, want_rr, hdr, resid, red, st);
        return launch_step_k<4, 16, 16>(P, g.zc, g.grid, m, j, mode, want_rr, hdr, resid, red, st);
    }
    if (m.tile == 2) return launch_step_k<3, 32, 16>(P, g.zc, g.grid, m, j, mode, want_rr, hdr, resid, red, st);
    if (m.tile == 1) return launch_step_k<3, 32, 8>(P, g.zc, g.grid, m, j, mode, want_rr, hdr, resid, red, st);
    return launch_step_k<3, 16, 16>(P, g.zc, g.grid, m, j, mode, want_rr, hdr, resid, red, st);
}

}  // namespace mpm
