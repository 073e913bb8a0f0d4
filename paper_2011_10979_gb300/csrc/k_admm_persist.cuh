// k_admm_persist.cuh -- persistent engine of the ADMM inner iteration (Sec. 3.1.1: eq. rpADMMI,
// eq. rpADMMII, eq. Zach-pADMM): one launch runs every inner iteration of one warp (linearisation)
// of a pyramid level, for one pair or a whole batch.
//
// Work: each pair's level is cut into segments -- strip sx (29 output columns, as in the streaming
// kernel k_admm_roll.cuh) by row band t of m (rows [t H / m, (t + 1) H / m), at least two rows
// each) -- and the host deals the segments out to the launch's warps so that every SM gets the
// same number of rows (usually one segment per warp, all warps resident in one wave).  A warp
// walks its segments with the streaming kernel's row pipeline (strip(), the same per-pixel
// arithmetic, so both engines give bitwise the same fields).
//
// Iterations: iteration k of a segment reads buffer (parity + k) & 1 and writes the other.  It
// needs, from the previous iteration, the fields within two rows above, one row below, two columns
// west and one east of its own outputs: those come only from the eight segments around it (row
// bands of at least two rows).  So instead of a grid-wide barrier each segment has a counter of
// finished iterations, which its warp publishes after finishing all its segments of an iteration
// (release: fence, then relaxed stores at GPU scope), and before iteration k each segment waits
// until its neighbours' counters reach k (relaxed loads, then an acquire fence).  The same wait
// covers the write-after-read hazard: a neighbour that finished iteration k - 1 has read
// everything it needs from the buffer this segment now overwrites.  A warp publishes an
// iteration only when it has finished it for all its segments, so the warp furthest behind only
// ever waits on counters that are already published: no cycle of waits can form.
//
// Stopping test (tolerance > 0, every 10th iteration): each segment stores its FP64 residual
// partial and arrives at its pair's counter; every warp of the pair waits for all of the pair's
// segments, sums the pair's partials in the same fixed order (so every warp takes the same
// decision) and, if the residual is below the tolerance, stops iterating that pair and sets its
// stop flag to the number of the check (non-zero: stopped; the number tells a warp that comes
// to the same check late that the pair stopped at this check, not before it).  The warp owning
// the pair's first segment adds the 10 iterations to the pair's count and records the residual.
//
// Every wait is bounded (wait_ns of %globaltimer): a wait that runs out marks the pair's timeout
// flag and the warp returns, so a lost arrival ends the launch with an error instead of a hang.
// All warps must be resident at once for the waits to end; the host sizes the grid to the
// co-resident capacity of the instance.
#pragma once
#include "k_admm_roll.cuh"

namespace tvl1 {
namespace persist {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(unsigned *p, unsigned v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Spins (all lanes) until pred() holds on every lane or wait_ns elapse; then an acquire fence.
// Returns false when the wait ran out.
template <typename Pred> __device__ __forceinline__ bool bounded_wait(Pred pred, long long wait_ns) {
    const unsigned long long t0 = now_ns();
    for (unsigned spins = 1;; ++spins) {
        if (__all_sync(FULL, pred())) break;
        if ((spins & 31) == 0 && __any_sync(FULL, (long long)(now_ns() - t0) > wait_ns)) return false;
    }
    __syncwarp();
    fence_acq_rel();
    return true;
}

// The flag index of neighbour `lane` (lanes 0..8: (dx, dt) = (lane % 3 - 1, lane / 3 - 1)) of
// segment s, or -1 for lanes without one (itself, outside the pair, lanes >= 9).
__device__ __forceinline__ int neighbour(int s, const PSeg &sg, int S, int lane) {
    if (lane >= 9 || lane == 4) return -1;
    const int sx = sg.sx + lane % 3 - 1, t = sg.t + lane / 3 - 1;
    if (sx < 0 || sx >= S || t < 0 || t >= sg.m) return -1;
    return s - (sg.t * S + sg.sx) + t * S + sx;
}

// Stopping test of every pair this warp holds segments of, at a checking iteration.  Returns
// false when a wait ran out (the pair's timeout flag is then set).
static __device__ __noinline__ bool check_pairs(const PersistArgs &A, int s_lo, int s_hi, unsigned round_) {
    const int lane = threadIdx.x & 31;
    // arrive once per held segment of a pair that is still iterating (its partial is stored)
    fence_acq_rel();
    __syncwarp();
    for (int q = s_lo; q < s_hi; ++q) {
        const int pair = A.segs[A.wseg[q]].pair;
        const int *done = A.pairs[pair].done;
        if (done && ld_relaxed((const unsigned *)done)) continue;
        if (lane == 0) atomicAdd(A.pbar + pair, 1u);
    }
    for (int q = s_lo; q < s_hi; ++q) {
        const int s = A.wseg[q];
        const int pair = A.segs[s].pair;
        bool seen = false;  // each pair once
        for (int q2 = s_lo; q2 < q; ++q2) seen |= A.segs[A.wseg[q2]].pair == pair;
        if (seen) continue;
        const PairScalars &P = A.scal[pair];
        const unsigned d = P.done ? ld_relaxed((const unsigned *)P.done) : 0u;
        if (d != 0u && d < round_) continue;  // stopped at an earlier check
        const unsigned need = (unsigned)(P.part_end - P.part_begin) * round_;
        if (!bounded_wait([&] { return ld_relaxed(A.pbar + pair) >= need; }, A.wait_ns)) {
            if (lane == 0 && P.timeout) *P.timeout = 1;
            return false;
        }
        // the pair's residual: lane-strided partial sums, then a fixed shuffle tree (same bits in
        // every warp of the pair)
        double v = 0.0;
        for (int k = P.part_begin + lane; k < P.part_end; k += 32) v += A.partials[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        const bool stop = A.tol > 0.0 && sqrt(v / P.rows) < A.tol;
        if (lane == 0) {
            bool lead = false;
            for (int q2 = s_lo; q2 < s_hi; ++q2) lead |= A.wseg[q2] == P.part_begin;
            if (lead) {
                *P.res_check = v;
                if (P.iters) *P.iters += 10;
            }
            if (stop && P.done) st_relaxed((unsigned *)P.done, round_);
        }
        __syncwarp();
    }
    return true;
}

// Three 128-thread blocks per SM: the run-time row loop of the beta > 0 instances needs about 168
// registers per lane; a cap of 128 (four blocks) spills some 450 bytes per lane.
#ifndef PERSIST_MIN_BLOCKS
#define PERSIST_MIN_BLOCKS 3
#endif

template <typename T, typename TF, bool HAS_W, int VARIANT>
__global__ void __launch_bounds__(roll::WARPS * 32, PERSIST_MIN_BLOCKS) k_admm_persist(PersistArgs A) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * roll::WARPS + (threadIdx.x >> 5);
    if (gw >= A.nwarps) return;
    const int s_lo = A.woff[gw], s_hi = A.woff[gw + 1];
    const int order[10] = {F_P1, F_P2, F_Q11, F_Q12, F_Q21, F_Q22, F_S, F_W, F_U, F_V};
    for (int it = 0; it < A.iters; ++it) {
        const bool checking = A.check && (it + 1) % 10 == 0;
        const bool want_res = checking || (A.final_res && it == A.iters - 1);
        for (int q = s_lo; q < s_hi; ++q) {
            const int s = A.wseg[q];
            const PSeg sg = A.segs[s];
            const PairIter *pp = A.pairs + sg.pair;
            if (pp->done && ld_relaxed((const unsigned *)pp->done)) continue;  // the pair stopped
            const int4 gq = *reinterpret_cast<const int4 *>(&pp->g);
            const int H = gq.x, W = gq.y, P = gq.z;
            const int S = (W + roll::SW - 1) / roll::SW;
            if (it > 0) {
                const int nb = neighbour(s, sg, S, lane);
                if (!bounded_wait([&] { return nb < 0 || ld_relaxed(A.flags + nb) >= (unsigned)it; }, A.wait_ns)) {
                    if (lane == 0 && A.scal[sg.pair].timeout) *A.scal[sg.pair].timeout = 1;
                    return;
                }
            }
            const Fields *in = pp->buf + ((A.parity + it) & 1), *out = pp->buf + ((A.parity + it + 1) & 1);
            const void *src[13];
            void *dst[10];
#pragma unroll
            for (int k = 0; k < 10; ++k) src[k < 7 ? k : k + 3] = in->f[order[k]];
#pragma unroll
            for (int k = 0; k < 10; ++k) dst[k] = out->f[k];
            src[7] = pp->Ix;
            src[8] = pp->Iy;
            src[9] = pp->It;
            const StepK SK = step_coefs(A.k, a_tilde_of(A.k, pp->ms_max), c_of(A.k, pp->ms_max));
            const int r0 = (int)((long long)sg.t * H / sg.m), r1 = (int)((long long)(sg.t + 1) * H / sg.m);
            const int c0 = sg.sx * roll::SW - 2;
            const bool interior = c0 >= 1 && c0 + 32 <= W - 1 && r0 >= 2 && r1 <= H - 2;
            const float res =
                interior
                    ? roll::strip<T, TF, HAS_W, VARIANT, 0, true>(src, dst, H, W, P, c0, r0, lane, A.k, pp->ms_max,
                                                                  r1 - r0, &SK)
                    : roll::strip<T, TF, HAS_W, VARIANT, 0, false>(src, dst, H, W, P, c0, r0, lane, A.k, pp->ms_max,
                                                                   r1 - r0, &SK);
            if (want_res) {
                double v = (double)res;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
                if (lane == 0) A.partials[s] = v;
            }
        }
        // publish once per iteration: this warp's stores of all its segments, then their
        // finished-iteration counters (a warp holding many segments pays one fence)
        fence_acq_rel();
        __syncwarp();
        if (lane == 0)
            for (int q = s_lo; q < s_hi; ++q) {
                const int s = A.wseg[q];
                if (s != A.withhold) st_relaxed(A.flags + s, (unsigned)(it + 1));
            }
        if (checking && !check_pairs(A, s_lo, s_hi, (unsigned)((it + 1) / 10))) return;
    }
}

template <typename T, typename TF, bool HAS_W, int VARIANT> __host__ void *kernel_of() {
    return (void *)k_admm_persist<T, TF, HAS_W, VARIANT>;
}

// The kernel instance of a method variant and storage pair.
template <typename T, typename TF> void *instance(const Coefs &k) {
    const bool has_w = k.beta != 0.f;
    const int v = (k.method == 1 ? 1 : 0) | (k.a_tilde_mode == 1 ? 2 : 0);
    switch (v) {
    case 0: return has_w ? kernel_of<T, TF, true, 0>() : kernel_of<T, TF, false, 0>();
    case 1: return has_w ? kernel_of<T, TF, true, 1>() : kernel_of<T, TF, false, 1>();
    case 2: return has_w ? kernel_of<T, TF, true, 2>() : kernel_of<T, TF, false, 2>();
    default: return has_w ? kernel_of<T, TF, true, 3>() : kernel_of<T, TF, false, 3>();
    }
}

}  // namespace persist
}  // namespace tvl1
