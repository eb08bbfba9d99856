// Batched persistent launch of the split step over many lattices.
//
// A batch advances a set of independent lattices (same DdQq and storage,
// any grid, parameters, walls and store layout each) with two launches per
// time step for the whole set.  Work items are blocks of kSplitThreads
// consecutive sites of one lattice; the grid is persistent (a fixed number
// of blocks per SM, each looping over items), so one captured CUDA graph of
// K steps stays valid while lattices join and leave: membership lives in a
// device table that the host rewrites between graph launches.
//
// Table: BatchHeader, then members sorted by the number of steps they take
// in the chunk (descending).  Launch k of the chunk (0 <= k < K) covers the
// first active[k] items: exactly the members with take > k.  An item is
// `span` consecutive blocks of kSplitThreads sites of one member (span is in
// the header: a longer item pays the member lookup and the argument loads
// once for more sites, a shorter one balances small members better; the
// batch autotuner picks it).
#pragma once

#include "lbm_split.cuh"

namespace lbm {

template <class R, class S>
struct BatchMember {
    SplitArgs<R, S> a[2];    // [k & 1]: arguments of the member's 1st, 2nd, ... step of the chunk
    int mode[2];             // stream mode of those steps (ping-pong, AA odd/even)
    long long first_item;    // prefix over members
    long long items;
    int take;                // steps in this chunk
    int has_mask;
};

// Member owning item t (first_item ascending, t < total items).
template <class R, class S>
__device__ __forceinline__ int batch_find(const BatchMember<R, S> *__restrict__ mem, int nmem, long long t)
{
    int lo = 0, hi = nmem - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (mem[mid].first_item <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <class L, class R, class C, int PHASE, bool HAS_MASK, int MODE>
__device__ __forceinline__ void batch_site(const SplitArgs<R, typename C::S> &a, int idx)
{
    // members have Q N < 2^32 (checked when they join): 32-bit indices
    if constexpr (PHASE == 0) moments_site<L, R, C, HAS_MASK, MODE, uint32_t>(a, idx);
    else collide_site<L, R, C, HAS_MASK, MODE, uint32_t>(a, idx);
}

// FP32 D2Q9 (4-byte storage, no stochastic rounding of a rest population):
// the site code reads the member's arguments from the table (read-only,
// cached) instead of a copy held in registers through the item, which lets
// the kernels run at 96 registers without spills, 5 blocks per SM (6 for the
// moments) instead of 4.  The others copy the arguments into registers per
// item and run 4 blocks per SM with FP32 arithmetic (128 registers; the
// collision spills a little, which costs less than a fourth of the warps: a
// batch of eight 128^3 D3Q27 lattices ran 2-5 % faster than at 3 blocks and
// 168 registers), 3 with FP64 (at 4 its site code spills kilobytes).
// Read by reference, or staged in shared memory, their site code needed
// more registers or ran slower.
template <class L, class R, class C>
inline constexpr bool kBatchArgsByRef = kPacked<R> && L::Q == 9 && !C::kRound16;

template <class L, class R, class C, int PHASE>
constexpr int batch_min_blocks()
{
    return kBatchArgsByRef<L, R, C> ? (PHASE == 1 ? 5 : 6) : (kPacked<R> ? 4 : 3);
}

// The item t of member j (base: its first site for this thread) in PHASE.
// PP: every member of the chunk uses the ping-pong store, so only that
// stream mode's code is compiled in.
template <class L, class R, class C, int PHASE, bool PP>
__device__ __forceinline__ void batch_item(const SplitArgs<R, typename C::S> &a, int mode, bool masked,
                                           long long base, int span)
{
    if constexpr (PHASE == 2) {
        if (!a.k.coupling) return;
        for (int s = 0; s < span; ++s) {
            const long long lidx = base + (long long)s * kSplitThreads;
            if (lidx >= a.N) break;
            if (masked) coupling_site<L, R, C, true, uint32_t>(a, (int)lidx);
            else coupling_site<L, R, C, false, uint32_t>(a, (int)lidx);
        }
    } else {
        for (int s = 0; s < span; ++s) {
            const long long lidx = base + (long long)s * kSplitThreads;
            if (lidx >= a.N) break;   // past the member's last site (so are the item's later blocks)
            const int idx = (int)lidx;
            if constexpr (PP) {
                if (masked) batch_site<L, R, C, PHASE, true, kPingPong>(a, idx);
                else batch_site<L, R, C, PHASE, false, kPingPong>(a, idx);
            } else if (masked) {
                if (mode == kPingPong) batch_site<L, R, C, PHASE, true, kPingPong>(a, idx);
                else if (mode == kAAOdd) batch_site<L, R, C, PHASE, true, kAAOdd>(a, idx);
                else batch_site<L, R, C, PHASE, true, kAAEven>(a, idx);
            } else {
                if (mode == kPingPong) batch_site<L, R, C, PHASE, false, kPingPong>(a, idx);
                else if (mode == kAAOdd) batch_site<L, R, C, PHASE, false, kAAOdd>(a, idx);
                else batch_site<L, R, C, PHASE, false, kAAEven>(a, idx);
            }
        }
    }
}

// PHASE 0: S0 + S1 of every member; PHASE 1: S0 + S2..S5; PHASE 2 (between
// the two, when some member takes it): the u^{n+1} coupling's omega-term of
// P^{n+1} for those members.
template <class L, class R, class C, int PHASE, bool PP = false>
__global__ void __launch_bounds__(kSplitThreads, batch_min_blocks<L, R, C, PHASE>())
    batch_kernel(const BatchHeader *__restrict__ hdr, const BatchMember<R, typename C::S> *__restrict__ mem, int k)
{
    using S = typename C::S;
    const int nmem = (int)hdr->nmem;
    const long long total = hdr->active[k];
    const int span = (int)hdr->span;
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
        const int j = batch_find(mem, nmem, t);
        const int q = k & 1;
        const int mode = mem[j].mode[q];
        const bool masked = mem[j].has_mask != 0;
        const long long base = (t - mem[j].first_item) * span * kSplitThreads + threadIdx.x;
        if constexpr (kBatchArgsByRef<L, R, C>) {
            batch_item<L, R, C, PHASE, PP>(mem[j].a[q], mode, masked, base, span);
        } else {
            SplitArgs<R, S> a = mem[j].a[q];
            a.seed += (unsigned)(k - q);   // a[q] holds the chunk's first steps; step k of the chunk
            batch_item<L, R, C, PHASE, PP>(a, mode, masked, base, span);
        }
    }
}

}  // namespace lbm
