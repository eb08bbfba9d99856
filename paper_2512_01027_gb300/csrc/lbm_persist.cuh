// Persistent split step: the two phases of the split form (moments, then
// stencils + collisions) in one launch per time step, so that what the
// moments phase hands to the collision phase (packed (u, phi) words, the
// second moments of g, the pulled h a second time) is still in L2 when it is
// read.
//
// Work items are kPersistSpan x kSplitThreads consecutive sites of one z-plane.
// Blocks take items from a ticket counter in this order of plane units
// (M = moments, C = collision, lag G >= 1 planes):
//   M(0) .. M(G), then M(1 + G), C(1), M(2 + G), C(2), ..., C(nz - 1), C(0)
// C(z) needs the moments of planes z-1, z, z+1 (periodic wrap in z where the
// lattice is periodic), and every one of them comes earlier in the order;
// the lag lets those moments finish before C(z) is handed out.  A block
// holding ticket t only waits for items with smaller tickets, which are held
// by blocks already running, so the waits end; each wait is still bounded,
// and the first one to run out sets an abort flag that ends every other wait
// at once and reports the timeout.
//
// Memory order: a moments block writes its outputs, every thread fences, the
// block counts itself done in mdone[plane]; a collision block's waiting
// thread observes the count (a volatile read) and fences, and the block
// barrier orders its other threads after that acquire.  Their loads of what
// other blocks wrote in this launch are then plain loads: no SM reads those
// lines earlier in the launch, so no L1 holds a stale copy.  (L2-only loads
// there were 2 % slower.)
#pragma once

#include "lbm_split.cuh"

namespace lbm {

struct PersistArgs {
    int *ctl;       // [0] ticket counter, [1] abort flag, [2 ..] moments items done per plane
    int nz;         // planes
    int bpp;        // work items per plane
    int nxy;        // sites per plane
    int zper;       // periodic in z
    int lag;        // planes by which the collisions trail the moments (>= 1)
    int stall;      // testing aid: moments of this plane are not counted (-1: none)
    int *err;       // bit 0 non-finite, bit 1 a dependency wait ran out
};

constexpr long long kPersistMaxSpin = 1LL << 26;            // polls, a backstop to the time limit
constexpr unsigned long long kPersistWaitNs = 1000000000ull;   // 1 s of waiting per plane

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr int kPersistLag = 2;
constexpr int kPersistSpan = 2;   // consecutive 128-site blocks per work item

// Plane unit u of the schedule: phase 0 = moments, 1 = collision.
__device__ __forceinline__ void persist_unit(int u, int nz, int lag, int &phase, int &plane)
{
    const int A = min(lag + 1, nz);          // leading moments units M(0) .. M(A - 1)
    const int K2 = max(0, nz - 1 - lag);     // z = 1 .. K2 come as pairs M(z + lag), C(z)
    if (u < A) {
        phase = 0;
        plane = u;
        return;
    }
    const int v = u - A;
    if (v < 2 * K2) {
        const int z = 1 + v / 2;
        phase = v & 1;
        plane = phase == 0 ? z + lag : z;
        return;
    }
    const int w = v - 2 * K2;                // single collision units C(K2 + 1) .. C(nz - 1), then C(0)
    phase = 1;
    plane = (w < nz - 1 - K2) ? K2 + 1 + w : 0;
}

// Wait until the moments of planes z-1, z, z+1 are complete.  Returns 0 if
// the wait was abandoned (timeout here or elsewhere).  The three counters are
// read together first: usually they are already complete.
__device__ __forceinline__ int persist_wait(const PersistArgs &p, int z)
{
    volatile int *ctl = p.ctl;
    int zz[3];
    bool need[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        zz[k] = z + k - 1;
        need[k] = true;
        if (zz[k] < 0 || zz[k] >= p.nz) {
            need[k] = p.zper != 0;
            zz[k] = (zz[k] + p.nz) % p.nz;
        }
    }
    const int c0 = ctl[2 + zz[0]], c1 = ctl[2 + zz[1]], c2 = ctl[2 + zz[2]];
    if ((!need[0] || c0 >= p.bpp) && c1 >= p.bpp && (!need[2] || c2 >= p.bpp)) {
        __threadfence();
        return 1;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (!need[k]) continue;
        long long it = 0;
        const unsigned long long t0 = global_ns();
        while (ctl[2 + zz[k]] < p.bpp) {
            if (ctl[1]) return 0;
            if (++it > kPersistMaxSpin || global_ns() - t0 > kPersistWaitNs) {
                atomicExch(p.ctl + 1, 1);
                atomicOr(p.err, 2);
                return 0;
            }
            __nanosleep(64);
        }
    }
    __threadfence();
    return 1;
}

template <class L, class C, bool HAS_MASK, int MODE>
__global__ void __launch_bounds__(kSplitThreads, kSplitMinBlocks)
    split_persistent_kernel(const SplitArgs<float, typename C::S> a, const PersistArgs p)
{
    __shared__ int s_t;
    __shared__ int s_ok;
    const int total = 2 * p.nz * p.bpp;
    for (;;) {
        if (threadIdx.x == 0) s_t = atomicAdd(p.ctl, 1);
        __syncthreads();
        const int t = s_t;
        __syncthreads();
        if (t >= total) break;
        const int unit = t / p.bpp, blk = t - unit * p.bpp;
        int phase, plane;
        persist_unit(unit, p.nz, p.lag, phase, plane);
        if (phase == 0) {
            for (int k = 0; k < kPersistSpan; ++k) {
                const int off = (blk * kPersistSpan + k) * kSplitThreads + (int)threadIdx.x;
                if (off < p.nxy) moments_site<L, float, C, HAS_MASK, MODE, uint32_t>(a, plane * p.nxy + off);
            }
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0 && plane != p.stall) atomicAdd(p.ctl + 2 + plane, 1);
        } else {
            if (threadIdx.x == 0) s_ok = persist_wait(p, plane);
            __syncthreads();
            if (s_ok)
                for (int k = 0; k < kPersistSpan; ++k) {
                    const int off = (blk * kPersistSpan + k) * kSplitThreads + (int)threadIdx.x;
                    if (off < p.nxy)
                        collide_site<L, float, C, HAS_MASK, MODE, uint32_t>(a, plane * p.nxy + off);
                }
        }
    }
}

}  // namespace lbm
