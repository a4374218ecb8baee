// batch.cuh -- launches that serve several subjects at once (mpm_fit_batch
// with opts.graph = 2): one launch per phase of a Newton update covers every
// subject of a batch class.  Blocks [start[s], start[s + 1]) of such a launch
// belong to subject s; each kernel body sees them as its own grid (VGrid) and
// reduces per subject through the subject's own workspace, so the CG scalars
// stay per subject (last block done).  The per-subject arguments travel in
// the kernel parameter (up to kBatchMax subjects per launch), the TMA tensor
// maps included.  Internal.
#pragma once

#include "pcg_step.cuh"

namespace mpm {

constexpr int kBatchMax = 16;

template <class A>
struct Batch {
    A a[kBatchMax];
    unsigned start[kBatchMax + 1];
    int n;
};

struct JtvArgs {
    DevProblem P;
    int zc;
    unsigned gx, gy, gz;
    const float* y;
    float* w;
    double* jtv;
    Reduce red;
};

struct GradArgs {
    DevProblem P;
    const void* x;
    const float *y, *b1p, *b1m;
    float *g, *h;
    double* nll;
    Reduce red;
    unsigned* status;     // kStatusTimeout of the staged pass
};

struct InitArgs {
    DevProblem P;
    int zc;
    unsigned gx, gy, gz;
    const float *h, *w, *g, *y;
    float4* z0;
    double tol2;
    WsHeader* hdr;
    double* resid;
    Reduce red;
};

struct StepArgs {
    CUtensorMap tz, tv, tp, tw, th, tx, tp2;
    DevProblem P;
    int nchunk, j, want_rr;
    float4 *zout, *vout, *pout, *xacc;
    WsHeader* hdr;
    double* resid;
    Reduce red;
    long long wait_cycles;
    int withhold;
};

struct FinalArgs {
    long long N;
    SolveBufs B;
    float *delta, *y_update;
    const WsHeader* hdr;
    double* report_rel;
    int* report_it;
};

struct UncArgs {
    DevProblem P;
    const float *h, *w, *y;
    float *var, *logdet, *moments;
    unsigned* status;
};

// kernel parameters are limited to 32764 bytes
static_assert(sizeof(Batch<StepArgs>) <= 32764, "kernel parameter space");
static_assert(sizeof(Batch<JtvArgs>) <= 32764, "kernel parameter space");
static_assert(sizeof(Batch<GradArgs>) <= 32764, "kernel parameter space");
static_assert(sizeof(Batch<InitArgs>) <= 32764, "kernel parameter space");
static_assert(sizeof(Batch<FinalArgs>) <= 32764, "kernel parameter space");
static_assert(sizeof(Batch<UncArgs>) <= 32764, "kernel parameter space");

// The batch of n subjects with blocks[s] hardware blocks each.
template <class A>
inline void fill_batch(Batch<A>& b, const A* a, const unsigned* blocks, int n)
{
    b.n = n;
    b.start[0] = 0;
    for (int s = 0; s < n; ++s) {
        b.a[s] = a[s];
        b.start[s + 1] = b.start[s] + blocks[s];
    }
}

}  // namespace mpm
