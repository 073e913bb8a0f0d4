// tvl1_plan.h -- the device arena layout of one pair's solve (its pyramid, state buffers,
// linearisation data, scratch, partial sums and device scalars) and the small helpers that turn
// solver parameters into kernel coefficients.  Shared by the whole-solve runtime (tvl1_api.cu)
// and the stage-by-stage solver of the serving loop (tvl1_step.cu).  Internal, not part of the C
// ABI.
#pragma once
#include <math.h>
#include <stddef.h>

#include "../../include/tvl1flow.h"
#include "tvl1_internal.h"

namespace tvl1 {

constexpr int MAX_LEVELS = 16;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline int level_size(int n, float eta) {
    int m = (int)floor((double)n * (double)eta + 0.5);
    return m < 1 ? 1 : m;
}

// Row pitch in elements: a multiple of 64 elements (>= 128 bytes for every storage type).
inline int pitch_of(int W) { return (int)align_up((size_t)W, 64); }

struct Plan {
    int L = 0, out_level = 0, prec = PREC_F32, pflow = PREC_F32;  // storage of duals/data, of w u v
    bool use32_last = false;
    int H[MAX_LEVELS], W[MAX_LEVELS], P[MAX_LEVELS];
    size_t plane32 = 0, planeT = 0;  // bytes of one finest-size plane in FP32 / storage precision
    size_t planeS = 0;               // stride of the state planes (fits both storage types)
    size_t img0[MAX_LEVELS], img1[MAX_LEVELS];
    size_t I1x, I1y, blur, stA, stB, stA32, stB32, data, data32, tmp, partials, misc, out;
    int max_blocks = 0;
    size_t total = 0;
};

// Device scalars at plan.misc.  c_cur sits directly before ms_max: kernels that are handed a
// pair's ms_max pointer read the adapted ADMM step c at ms_max[-1] (Coefs::c_dev); ms_max and
// done are adjacent so that one 8-byte memset clears both at the start of a warp.
struct Misc {
    float c_cur;
    float ms_max;
    int done;
    long long iters;
    double res_check, res_final, energy, dual;
    int timeout;  // a bounded wait of the persistent engine ran out
};
static_assert(offsetof(Misc, ms_max) == offsetof(Misc, c_cur) + sizeof(float), "c_cur must precede ms_max");
static_assert(offsetof(Misc, done) == offsetof(Misc, ms_max) + sizeof(float), "done must follow ms_max");

// The arena layout of one H x W pair with these parameters (offsets from the pair's base).
Plan make_plan(int H, int W, const of_params *p);

// Kernel coefficients of the parameters.
Coefs coefs_of(const of_params *p);

// The 13 planes of a state buffer at `base`, `plane` bytes apart.
Fields fields_at(char *base, size_t plane);

inline Geom geom_of(const Plan &pl, int l) { return Geom{pl.H[l], pl.W[l], pl.P[l]}; }

}  // namespace tvl1
