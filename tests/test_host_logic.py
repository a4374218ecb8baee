"""The library's host-side decisions on the CPU: the server's arena and
admission pick, the lanes of a batched graph and the z split of the TMA
PCG iteration.  They live in csrc/host_logic.h, which needs no CUDA; a small C++
harness compiled here with g++ exposes them through ctypes, and every check
below is a property the decision must have, under seeded random inputs."""
import ctypes
import os
import random
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2102_01604_gb300", "csrc")
HARNESS = os.path.join(ROOT, "tests", "host_logic_harness.cpp")

BIG = 1 << 21          # voxels at which one fit keeps the GPU busy
ULL = ctypes.c_size_t
LL = ctypes.c_longlong


@pytest.fixture(scope="module")
def hl(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("host_logic") / "libhl.so")
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-Werror", "-shared", "-fPIC",
                    "-I", CSRC, HARNESS, "-o", so], check=True)
    h = ctypes.CDLL(so)
    h.hl_gpu_load.restype = ctypes.c_double
    h.hl_gpu_load.argtypes = [LL]
    h.hl_max_load.restype = ctypes.c_double
    h.hl_arena_new.restype = ctypes.c_void_p
    h.hl_arena_new.argtypes = [ULL]
    h.hl_arena_delete.argtypes = [ctypes.c_void_p]
    h.hl_arena_alloc.argtypes = [ctypes.c_void_p, ULL, ctypes.POINTER(ULL)]
    h.hl_arena_release.argtypes = [ctypes.c_void_p, ULL, ULL]
    h.hl_arena_largest.restype = ULL
    h.hl_arena_largest.argtypes = [ctypes.c_void_p]
    h.hl_arena_blocks.argtypes = [ctypes.c_void_p, ctypes.POINTER(ULL), ctypes.POINTER(ULL), ctypes.c_int]
    h.hl_lane_plan.argtypes = [ctypes.c_int, ctypes.POINTER(LL), ctypes.c_char_p,
                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    h.hl_tma_chunks.argtypes = [LL, ctypes.c_int, LL]
    h.hl_share_wave.restype = LL
    h.hl_share_wave.argtypes = [ctypes.c_int, ctypes.POINTER(LL), ctypes.POINTER(ctypes.c_int), LL,
                                ctypes.POINTER(LL), ctypes.POINTER(ctypes.c_int)]
    h.hl_admit_pick.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(LL), ctypes.POINTER(ULL),
                                ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_int,
                                ctypes.POINTER(ULL)]
    return h


def test_header_needs_no_cuda():
    text = open(os.path.join(CSRC, "host_logic.h")).read()
    includes = [l for l in text.splitlines() if l.startswith("#include")]
    assert includes and not any("cuda" in l.lower() or ".cuh" in l for l in includes)


# ---------------------------------------------------------------- gpu load

def test_gpu_load(hl):
    assert hl.hl_gpu_load(0) == 0.0
    assert hl.hl_gpu_load(BIG // 2) == 0.5
    assert hl.hl_gpu_load(BIG - 1) < 1.0
    assert hl.hl_gpu_load(BIG) == 1.0 and hl.hl_gpu_load(1 << 30) == 1.0
    rng = random.Random(3)
    xs = sorted(rng.randrange(0, 1 << 23) for _ in range(500))
    ys = [hl.hl_gpu_load(x) for x in xs]
    assert all(a <= b for a, b in zip(ys, ys[1:]))
    assert hl.hl_max_load() == 1.5


# ---------------------------------------------------------------- arena

class ArenaView:
    def __init__(self, hl, nbytes):
        self.hl, self.nbytes = hl, nbytes
        self.a = hl.hl_arena_new(nbytes)

    def blocks(self):
        n = self.hl.hl_arena_blocks(self.a, None, None, 0)
        offs, sizes = (ULL * max(n, 1))(), (ULL * max(n, 1))()
        assert self.hl.hl_arena_blocks(self.a, offs, sizes, n) == n
        return [(offs[i], sizes[i]) for i in range(n)]

    def alloc(self, n):
        off = ULL(0)
        ok = self.hl.hl_arena_alloc(self.a, n, ctypes.byref(off))
        return off.value if ok else None

    def release(self, off, n):
        self.hl.hl_arena_release(self.a, off, n)

    def largest(self):
        return self.hl.hl_arena_largest(self.a)

    def close(self):
        self.hl.hl_arena_delete(self.a)


def round256(n):
    return (n + 255) // 256 * 256


def check_arena(ar, live):
    free = ar.blocks()
    # free blocks: non-empty, sorted, coalesced (no two touch)
    assert all(s > 0 for _, s in free)
    assert all(o1 + s1 < o2 for (o1, s1), (o2, _) in zip(free, free[1:]))
    # free blocks and live allocations tile [0, bytes) with no overlap
    spans = sorted(free + [(o, round256(n)) for o, n in live.items()])
    pos = 0
    for o, s in spans:
        assert o == pos, (o, pos)
        pos = o + s
    assert pos == ar.nbytes
    assert ar.largest() == max((s for _, s in free), default=0)


@pytest.mark.parametrize("seed", range(4))
def test_arena_first_fit_no_overlap_and_coalescing(hl, seed):
    rng = random.Random(seed)
    nbytes = 256 * rng.randrange(64, 4096)
    ar = ArenaView(hl, nbytes)
    live = {}
    try:
        for _ in range(600):
            if live and rng.random() < 0.45:
                off = rng.choice(sorted(live))
                ar.release(off, live.pop(off))
            else:
                n = rng.choice([1, 255, 256, 257, rng.randrange(1, nbytes // 4)])
                before = ar.blocks()
                off = ar.alloc(n)
                fitting = [o for o, s in before if s >= round256(n)]
                if off is None:
                    assert not fitting
                else:
                    assert off == fitting[0] and off % 256 == 0   # first fit, aligned
                    live[off] = n
            check_arena(ar, live)
        for off in rng.sample(sorted(live), len(live)):
            ar.release(off, live.pop(off))
            check_arena(ar, live)
        assert ar.blocks() == [(0, nbytes)]
    finally:
        ar.close()


def test_arena_ragged_size(hl):
    ar = ArenaView(hl, 1000)          # not a multiple of 256
    try:
        assert ar.alloc(1000) is None  # rounds to 1024
        assert ar.alloc(768) == 0
        assert ar.alloc(1) is None     # 232 bytes left, a request takes 256
        ar.release(0, 768)
        assert ar.blocks() == [(0, 1000)]
    finally:
        ar.close()


# ---------------------------------------------------------------- lanes

def lane_plan(hl, voxels, empty=None):
    n = len(voxels)
    empty = empty or [False] * n
    lane, pos = (ctypes.c_int * n)(), (ctypes.c_int * n)()
    nl = hl.hl_lane_plan(n, (LL * n)(*voxels), bytes(1 if e else 0 for e in empty), lane, pos)
    lanes = [[] for _ in range(nl)]
    for i in range(n):
        if lane[i] >= 0:
            lanes[lane[i]].append((pos[i], i))
    return [[i for _, i in sorted(l)] for l in lanes]


def test_lane_plan_examples(hl):
    M = 1 << 20
    # one large subject: the small ones share a single lane beside it (0.5 left)
    assert lane_plan(hl, [4 * M, M, M, M // 2, M // 4]) == [[0], [1, 2, 3, 4]]
    # all small, each 0.5 or 0.25: three lanes keep 1.5; largest first, round robin
    assert lane_plan(hl, [M, M, M // 2, M // 2]) == [[0, 3], [1], [2]]
    # tiny subjects: one lane each
    assert lane_plan(hl, [1 << 16] * 8) == [[i] for i in range(8)]
    # only large ones: one lane, in the caller's order
    assert lane_plan(hl, [3 * BIG, BIG, 2 * BIG]) == [[0, 1, 2]]
    # empty subjects are left out
    assert lane_plan(hl, [M, 0, M], [False, True, False]) == [[0], [2]]
    assert lane_plan(hl, []) == [] and lane_plan(hl, [7], [True]) == []


@pytest.mark.parametrize("seed", range(6))
def test_lane_plan_properties(hl, seed):
    rng = random.Random(100 + seed)
    for _ in range(200):
        n = rng.randrange(1, 24)
        voxels = [rng.choice([rng.randrange(1, 1 << 16), rng.randrange(1, BIG), rng.randrange(BIG, 4 * BIG)])
                  for _ in range(n)]
        empty = [rng.random() < 0.1 for _ in range(n)]
        lanes = lane_plan(hl, voxels, empty)
        placed = sorted(i for l in lanes for i in l)
        assert placed == [i for i in range(n) if not empty[i]]       # each subject once
        large = [i for i in placed if voxels[i] >= BIG]
        small = [i for i in placed if voxels[i] < BIG]
        if large:
            assert lanes[0] == large                                  # one lane, in order
        small_lanes = lanes[1:] if large else lanes
        assert all(voxels[i] < BIG for l in small_lanes for i in l)
        assert all(lanes)                                              # no empty lane
        if not small:
            assert len(lanes) == (1 if large else 0)
            continue
        for l in small_lanes:                                         # largest first
            assert all(voxels[a] >= voxels[b] for a, b in zip(l, l[1:]))
        sizes = [len(l) for l in small_lanes]
        assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1      # dealt round robin
        budget = 0.5 if large else 1.5
        top = max(hl.hl_gpu_load(voxels[i]) for i in small)
        k = len(small_lanes)
        assert k == 1 or k * top <= budget + 1e-12                    # within the load budget
        assert k == len(small) or (k + 1) * top > budget - 1e-12     # and no more serial than needed


# ---------------------------------------------------------------- TMA z split

def chunk_cost(tiles, nz, wave, c):
    per = -(-nz // c)
    return -(-tiles * c // wave) * (per + 2)


@pytest.mark.parametrize("seed", range(3))
def test_tma_chunks(hl, seed):
    rng = random.Random(200 + seed)
    cases = [(165, 256, 304), (165, 256, 456), (44, 64, 304), (12, 3, 304), (1, 1, 152)]
    cases += [(rng.randrange(1, 2000), rng.randrange(1, 600), 152 * rng.randrange(1, 5)) for _ in range(300)]
    for tiles, nz, wave in cases:
        c = hl.hl_tma_chunks(tiles, nz, wave)
        allowed = [d for d in range(1, nz + 1) if d == 1 or -(-nz // d) >= 4]
        assert c in allowed
        assert chunk_cost(tiles, nz, wave, c) == min(chunk_cost(tiles, nz, wave, d) for d in allowed)
        # the kernel's balanced split [ch*nz/c, (ch+1)*nz/c) covers every plane once, no range empty
        bounds = [ch * nz // c for ch in range(c + 1)]
        assert bounds[0] == 0 and bounds[-1] == nz
        assert all(b > a for a, b in zip(bounds, bounds[1:]))


def share_wave(hl, tiles, nz, wave):
    n = len(tiles)
    b, c = (LL * n)(), (ctypes.c_int * n)()
    cost = hl.hl_share_wave(n, (LL * n)(*tiles), (ctypes.c_int * n)(*nz), wave, b, c)
    return cost, list(b), list(c)


def _splits(nz):
    return [d for d in range(1, nz + 1) if d == 1 or -(-nz // d) >= 4]


def _min_cost(tiles, nz, b):
    """Lowest rounds x (planes + 2) of one volume with b blocks."""
    return min(chunk_cost(tiles, nz, b, c) for c in _splits(nz))


@pytest.mark.parametrize("seed", range(4))
def test_share_wave_is_optimal(hl, seed):
    """Brute force over every assignment of blocks on small groups: the
    returned largest cost is the minimum, the returned shares reach it, sum
    to at most the wave and cannot lose a block without exceeding it."""
    import itertools
    rng = random.Random(500 + seed)
    for _ in range(40):
        n = rng.randrange(1, 4)
        tiles = [rng.randrange(1, 9) for _ in range(n)]
        nz = [rng.randrange(1, 24) for _ in range(n)]
        wave = rng.randrange(n, 14)
        best = min(max(_min_cost(t, z, b) for t, z, b in zip(tiles, nz, bs))
                   for bs in itertools.product(range(1, wave + 1), repeat=n) if sum(bs) <= wave)
        cost, blocks, chunks = share_wave(hl, tiles, nz, wave)
        assert cost == best, (tiles, nz, wave)
        assert sum(blocks) <= wave and min(blocks) >= 1
        for t, z, b, c in zip(tiles, nz, blocks, chunks):
            assert c in _splits(z)
            assert chunk_cost(t, z, b, c) <= cost
            assert b == 1 or _min_cost(t, z, b - 1) > cost


def test_share_wave_single_volume_is_the_solo_launch(hl):
    """One volume: the cost of the solo launch (tma_chunks over the whole wave)."""
    for tiles, nz, wave in [(180, 256, 304), (165, 256, 456), (16, 64, 304), (44, 64, 304)]:
        cost, blocks, chunks = share_wave(hl, [tiles], [nz], wave)
        c = hl.hl_tma_chunks(tiles, nz, wave)
        assert cost == chunk_cost(tiles, nz, wave, c)
        assert blocks[0] <= min(wave, tiles * c)


# ---------------------------------------------------------------- admission

def admit(hl, ar, queue, load, max_slots):
    """queue: list of (n_vox, ws_bytes, overtaken) in arrival order."""
    n = len(queue)
    off = ULL(0)
    i = hl.hl_admit_pick(ar.a, n, (LL * n)(*[q[0] for q in queue]), (ULL * n)(*[q[1] for q in queue]),
                         (ctypes.c_int * n)(*[q[2] for q in queue]), load, max_slots, ctypes.byref(off))
    return i, off.value


@pytest.mark.parametrize("seed", range(4))
def test_admit_pick_properties(hl, seed):
    rng = random.Random(300 + seed)
    max_slots = 4
    for _ in range(300):
        ar = ArenaView(hl, 256 * rng.randrange(16, 256))
        try:
            for _ in range(rng.randrange(0, 4)):   # some of the arena already taken
                ar.alloc(256 * rng.randrange(1, 32))
            free_before = ar.blocks()
            load = rng.choice([0.0, 0.25, 0.5, 1.0, 1.25])
            queue = [(rng.choice([1 << 16, 1 << 19, 1 << 20, BIG, 4 * BIG]), 256 * rng.randrange(1, 64),
                      rng.choice([0, 0, 0, 1, 2 * max_slots])) for _ in range(rng.randrange(1, 8))]
            i, off = admit(hl, ar, queue, load, max_slots)

            def fits(q):
                return load == 0.0 or load + hl.hl_gpu_load(q[0]) <= 1.5

            def room(q):
                return any(s >= round256(q[1]) for _, s in free_before)

            urgent = [j for j, q in enumerate(queue) if q[2] >= 2 * max_slots]
            if urgent:
                u = urgent[0]
                assert i == (u if fits(queue[u]) and room(queue[u]) else -1)
            elif i >= 0:
                assert fits(queue[i]) and room(queue[i])
                small = min((q[0] for q in queue if fits(q)))
                first_small = next(j for j, q in enumerate(queue) if fits(q) and q[0] == small)
                if i != first_small:   # the smallest had no room: first in arrival order with room
                    assert not room(queue[first_small])
                    assert i == next(j for j, q in enumerate(queue) if fits(q) and room(q))
            else:
                assert not any(fits(q) and room(q) for q in queue)
            if i >= 0:                 # the workspace was taken from the arena at off
                assert any(o <= off and off + round256(queue[i][1]) <= o + s for o, s in free_before)
                assert sum(s for _, s in ar.blocks()) == sum(s for _, s in free_before) - round256(queue[i][1])
            else:
                assert ar.blocks() == free_before
        finally:
            ar.close()


def test_admission_does_not_starve_a_large_request(hl):
    """A large request queued behind a steady stream of small ones: smallest
    first alone would pass it over for as long as small fits keep the GPU
    busy; aging admits it after 2 x max_slots overtakes."""
    max_slots = 4
    ar = ArenaView(hl, 1 << 30)
    try:
        queue = [[4 * BIG, 1 << 20, 0, "large"]]
        active = []   # [remaining ticks, n_vox, off, ws]
        admitted_large_at = None
        for tick in range(200):
            queue += [[BIG // 3, 1 << 16, 0, "small"] for _ in range(2)]
            for a in active:
                a[0] -= 1
            for a in [a for a in active if a[0] <= 0]:
                ar.release(a[2], a[3])
                active.remove(a)
            while len(active) < max_slots and queue:
                load = sum(hl.hl_gpu_load(a[1]) for a in active)
                i, off = admit(hl, ar, [tuple(q[:3]) for q in queue], load, max_slots)
                if i < 0:
                    break
                for q in queue[:i]:
                    q[2] += 1
                q = queue.pop(i)
                active.append([3, q[0], off, q[1]])
                if q[3] == "large":
                    admitted_large_at = tick
            assert sum(hl.hl_gpu_load(a[1]) for a in active) <= 1.5 or len(active) == 1
            if admitted_large_at is not None:
                break
        assert admitted_large_at is not None and admitted_large_at < 20
    finally:
        ar.close()
