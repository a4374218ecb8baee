// C entry points over the library's CUDA-free host logic (host_logic.h), so
// that tests/test_host_logic.py drives it through ctypes on the CPU.
#include <cstring>
#include <vector>

#include "host_logic.h"

using namespace mpm;

extern "C" {

double hl_gpu_load(long long n) { return gpu_load(n); }
double hl_max_load() { return kMaxLoad; }

void* hl_arena_new(size_t bytes)
{
    Arena* a = new Arena;
    a->init(nullptr, bytes);
    return a;
}
void hl_arena_delete(void* a) { delete static_cast<Arena*>(a); }
int hl_arena_alloc(void* a, size_t n, size_t* off) { return static_cast<Arena*>(a)->alloc(n, off) ? 1 : 0; }
void hl_arena_release(void* a, size_t off, size_t n) { static_cast<Arena*>(a)->release(off, n); }
size_t hl_arena_largest(void* a) { return static_cast<Arena*>(a)->largest(); }
// free blocks in offset order; returns how many there are (writes at most cap)
int hl_arena_blocks(void* a, size_t* offs, size_t* sizes, int cap)
{
    int i = 0;
    for (auto& f : static_cast<Arena*>(a)->free_) {
        if (i < cap) {
            offs[i] = f.first;
            sizes[i] = f.second;
        }
        ++i;
    }
    return i;
}

// lane_of[i] / pos[i]: lane and position of subject i (-1 when left out);
// returns the number of lanes
int hl_lane_plan(int n, const long long* voxels, const char* empty, int* lane_of, int* pos)
{
    const std::vector<std::vector<int>> lanes =
        lane_plan(std::vector<long long>(voxels, voxels + n), std::vector<char>(empty, empty + n));
    for (int i = 0; i < n; ++i) lane_of[i] = pos[i] = -1;
    for (int l = 0; l < (int)lanes.size(); ++l)
        for (int k = 0; k < (int)lanes[l].size(); ++k) {
            lane_of[lanes[l][k]] = l;
            pos[lanes[l][k]] = k;
        }
    return (int)lanes.size();
}

int hl_tma_chunks(long long tiles, int nz, long long wave) { return tma_chunks(tiles, nz, wave); }

long long hl_share_wave(int n, const long long* tiles, const int* nz, long long wave, long long* blocks,
                        int* chunks)
{
    std::vector<long long> b;
    std::vector<int> c;
    const long long cost = share_wave(std::vector<long long>(tiles, tiles + n),
                                      std::vector<int>(nz, nz + n), wave, b, c);
    for (int i = 0; i < n; ++i) {
        blocks[i] = b[i];
        chunks[i] = c[i];
    }
    return cost;
}

int hl_admit_pick(void* a, int n, const long long* n_vox, const size_t* ws, const int* overtaken,
                  double load, int max_slots, size_t* off)
{
    std::vector<Queued> q(n);
    for (int i = 0; i < n; ++i) q[i] = {n_vox[i], ws[i], overtaken[i]};
    return admit_pick(q, load, max_slots, *static_cast<Arena*>(a), off);
}

}  // extern "C"
