// host_logic.h -- host-side decisions of the library that make no CUDA call:
// the server's device arena and admission pick, the GPU-load rule shared by
// the server and the batched graph, the lanes of a batched graph, and the z
// split of the TMA PCG iteration.  Plain C++17, so the CPU tests compile and check it directly.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <iterator>
#include <map>
#include <vector>

namespace mpm {

// Share of the GPU one fit keeps busy: about 2^21 voxels keep every kernel of
// a fit at a full wave, so larger volumes count as 1, smaller ones pro rata.
inline double gpu_load(long long n_vox)
{
    return n_vox >= (1LL << 21) ? 1.0 : (double)n_vox / (double)(1LL << 21);
}

// Fits running side by side may keep at most this much of the GPU busy.
constexpr double kMaxLoad = 1.5;

// First-fit allocator over a caller-owned device range: offsets and sizes
// only, sizes rounded up to 256 bytes, free blocks kept sorted and coalesced.
struct Arena {
    char* base = nullptr;
    size_t bytes = 0;
    std::map<size_t, size_t> free_;   // offset -> size, coalesced

    void init(void* b, size_t n)
    {
        base = static_cast<char*>(b);
        bytes = n;
        free_.clear();
        if (n) free_[0] = n;
    }
    bool alloc(size_t n, size_t* off)
    {
        n = (n + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = (n + 255) & ~(size_t)255;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t largest() const
    {
        size_t m = 0;
        for (auto& f : free_) m = f.second > m ? f.second : m;
        return m;
    }
};

// One queued request as the fit server's admission sees it.
struct Queued {
    long long n_vox;      // volume size
    size_t ws_bytes;      // workspace it needs in the arena
    int overtaken;        // later requests admitted before it
};

// Admission pick of the fit server for one free slot.  `queue` is in arrival
// order and `load` the summed gpu_load of the active fits; a request fits the
// load when the GPU is idle or the sum stays within kMaxLoad.  A request
// overtaken by 2 x max_slots later ones comes first, and while it does not
// fit the load and the arena nothing is admitted.  Otherwise the smallest
// volume that fits the load (ties by arrival); when that one finds no room in
// the arena, the first in arrival order that fits both.  Returns the index
// into `queue`, its workspace already taken from `arena` at *off, or -1.
inline int admit_pick(const std::vector<Queued>& queue, double load, int max_slots,
                      Arena& arena, size_t* off)
{
    auto fits = [&](const Queued& c) { return load == 0.0 || load + gpu_load(c.n_vox) <= kMaxLoad; };
    const int n = (int)queue.size();
    for (int i = 0; i < n; ++i)
        if (queue[i].overtaken >= 2 * max_slots)
            return fits(queue[i]) && arena.alloc(queue[i].ws_bytes, off) ? i : -1;
    int pick = -1;
    for (int i = 0; i < n; ++i)
        if (fits(queue[i]) && (pick < 0 || queue[i].n_vox < queue[pick].n_vox)) pick = i;
    if (pick < 0) return -1;
    if (arena.alloc(queue[pick].ws_bytes, off)) return pick;
    for (int i = 0; i < n; ++i)
        if (fits(queue[i]) && arena.alloc(queue[i].ws_bytes, off)) return i;
    return -1;
}

// Lanes of a batched graph (each lane a chain of subjects run in order, all
// lanes side by side).  Subjects that fill the GPU on their own form one lane,
// first; the smaller ones, largest first, are dealt round-robin to as many
// lanes as keep the load of the lanes running together within 1.5 (0.5
// beside the large lane).  `voxels[i]` is subject i's size; empty subjects
// are left out, and so is a lane that would hold nothing.
inline std::vector<std::vector<int>> lane_plan(const std::vector<long long>& voxels,
                                               const std::vector<char>& empty)
{
    std::vector<int> large, small;
    double max_small = 0.0;
    for (int i = 0; i < (int)voxels.size(); ++i) {
        if (empty[i]) continue;
        const double l = gpu_load(voxels[i]);
        if (l >= 1.0) {
            large.push_back(i);
        } else {
            small.push_back(i);
            max_small = std::max(max_small, l);
        }
    }
    std::stable_sort(small.begin(), small.end(),
                     [&](int a, int b) { return voxels[a] > voxels[b]; });
    const double budget = large.empty() ? kMaxLoad : kMaxLoad - 1.0;
    int n_small = 0;
    if (!small.empty())
        n_small = std::max(1, std::min((int)std::floor(budget / max_small), (int)small.size()));
    std::vector<std::vector<int>> lanes;
    if (!large.empty()) lanes.push_back(large);
    for (int l = 0; l < n_small; ++l) lanes.emplace_back();
    for (size_t k = 0; k < small.size(); ++k)
        lanes[(large.empty() ? 0 : 1) + k % n_small].push_back(small[k]);
    return lanes;
}

// Number of z ranges of the TMA PCG iteration: the launch is one wave of `wave`
// resident blocks over tiles x nchunk items, block b taking items b, b + G,
// ...; nchunk minimises rounds x (planes per item + 2), so that the last
// round leaves few slots idle and items stay long enough that their two halo
// planes and the ring's start-up are small.  Planes per item count as
// ceil(nz / nchunk), and splits where that falls below 4 are not considered.
inline int tma_chunks(long long tiles, int nz, long long wave)
{
    int best = 1;
    long long best_cost = -1;
    for (int c = 1; c <= nz; ++c) {
        const long long per = (nz + c - 1) / c;
        if (per < 4 && c > 1) break;
        const long long rounds = (tiles * c + wave - 1) / wave;
        const long long cost = rounds * (per + 2);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = c;
        }
    }
    return best;
}

// Shares of one launch of the TMA PCG iteration between several volumes (a
// phase-batched group): volume s, of tiles[s] tiles per plane and nz[s]
// planes, gets blocks[s] blocks and chunks[s] z ranges.  Each of its blocks
// walks ceil(tiles c / blocks) items of ceil(nz / c) + 2 planes (splits of
// fewer than 4 planes are not considered, as in tma_chunks), so the launch
// lasts about the largest such cost among the volumes.  The shares minimise
// that largest cost with at least one block per volume and at most `wave`
// blocks in all (given n <= wave), each volume taking the fewest blocks that
// keep it within the minimum.  Returns the minimum.
inline long long share_wave(const std::vector<long long>& tiles, const std::vector<int>& nz,
                            long long wave, std::vector<long long>& blocks, std::vector<int>& chunks)
{
    const size_t n = tiles.size();
    blocks.assign(n, 1);
    chunks.assign(n, 1);
    if (n == 0) return 0;
    // fewest blocks that keep volume s within cost T, and the split for it
    // (-1: no split fits T)
    auto need = [&](size_t s, long long T, int* c_out) {
        long long best = -1;
        for (int c = 1; c <= nz[s]; ++c) {
            const long long per = (nz[s] + c - 1) / c;
            if (per < 4 && c > 1) break;
            const long long rounds = T / (per + 2);
            if (rounds < 1) continue;
            const long long b = (tiles[s] * c + rounds - 1) / rounds;
            if (best < 0 || b < best) {
                best = b;
                *c_out = c;
            }
        }
        return best;
    };
    auto fits = [&](long long T, bool keep) {
        long long sum = 0;
        for (size_t s = 0; s < n; ++s) {
            int c = 1;
            const long long b = need(s, T, &c);
            if (b < 0) return false;
            sum += b;
            if (keep) {
                blocks[s] = b;
                chunks[s] = c;
            }
        }
        return sum <= wave;
    };
    long long hi = 0;   // one block per volume, whole columns: always fits
    for (size_t s = 0; s < n; ++s) hi = std::max(hi, tiles[s] * (nz[s] + 2LL));
    if ((long long)n > wave) return hi;
    long long lo = 0;   // never fits
    while (hi - lo > 1) {
        const long long mid = lo + (hi - lo) / 2;
        if (fits(mid, false))
            hi = mid;
        else
            lo = mid;
    }
    fits(hi, true);
    return hi;
}

}  // namespace mpm
