// tvl1_step.h -- stage-by-stage solves (tvl1_step.cu) for the serving loop (tvl1_serve.cu): every
// call of step_run() advances each pair of a changing set by one warp of its current pyramid
// level, the inner iterations of all of them in shared launches.  Internal, not part of the C ABI.
#pragma once
#include <vector>

#include "tvl1_plan.h"

namespace tvl1 {

// One pair's solve in progress.  A points to a device region of step_pair_bytes() bytes laid out
// by its Plan; (l, wp) is the next stage; cur the state buffer holding the current state.
struct StepPair {
    char *A = nullptr;
    Plan pl;
    int H = 0, W = 0;
    int l = 0, wp = 0, cur = 0;
    int prec = PREC_F32, pflow = PREC_F32;  // storage of the current stage
    bool in32 = false;                      // the FP32 last-warp buffers are in use
    bool finished = false;                  // the output level is done; the flow is at pl.out
};

// Launch tables of a step: one device block (tables and partial sums) and a ring of pinned host
// staging buffers, each reused only after the copy from it has run.
struct StepTables {
    static constexpr int NSTAGE = 4;
    char *dev = nullptr;
    size_t dev_bytes = 0;
    char *host[NSTAGE] = {};
    size_t host_bytes[NSTAGE] = {};
    cudaEvent_t ev[NSTAGE] = {};
    int next = 0;
    ~StepTables();
};

size_t step_pair_bytes(int H, int W, const of_params *p);
void step_pair_init(StepPair &q, char *region, int H, int W, const of_params *p);
// Copies the H x W images in from pinned host memory (dense) and builds the pyramid, on s.
void step_pair_start(StepPair &q, const float *I0, const float *I1, const of_params *p, cudaStream_t s);
// Enqueues one stage of every pair in `act` on s; pairs whose output level is done get
// finished = true and their flow at pl.out.
cudaError_t step_run(std::vector<StepPair *> &act, const of_params *p, StepTables &T, cudaStream_t s);
// Copies a finished pair's flow (dense, out-level size) and its device scalars (a Misc) to host
// memory, on s.
void step_pair_finish(const StepPair &q, float *u, float *v, Misc *misc, cudaStream_t s);

}  // namespace tvl1
