// Host side of the batched persistent launch (lbm_batch_*) and of the
// autotuner (lbm_autotune).
#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "lbm_internal.h"

using namespace lbm;

namespace {

int bfail(lbm_batch_ctx *b, int code, const std::string &msg)
{
    if (b) b->err = msg;
    return code;
}

int bcuda(lbm_batch_ctx *b, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return LBM_OK;
    b->err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

void drop_graphs(lbm_batch_ctx *b)
{
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.second);
    b->graphs.clear();
}

// Device and pinned host tables for at least `members` members.
int ensure_table(lbm_batch_ctx *b, size_t members)
{
    if (members <= b->cap_members && b->d_table) return LBM_OK;
    size_t cap = std::max<size_t>(16, b->cap_members);
    while (cap < members) cap *= 2;
    const size_t bytes = batch_header_bytes() + cap * b->ops->batch_member_bytes();
    cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    if (b->d_table) cudaFree(b->d_table);
    if (b->h_table) cudaFreeHost(b->h_table);
    b->d_table = nullptr;
    b->h_table = nullptr;
    b->cap_members = 0;
    b->table_bytes = 0;
    int rc = bcuda(b, cudaMalloc(&b->d_table, bytes), "cudaMalloc(batch table)");
    if (rc == LBM_OK) rc = bcuda(b, cudaMallocHost(&b->h_table, bytes), "cudaMallocHost(batch table)");
    if (rc != LBM_OK) return rc;
    std::memset(b->h_table, 0, bytes);
    b->cap_members = cap;
    b->table_bytes = bytes;
    return LBM_OK;
}

// Executable graph of one chunk of K steps: table upload + 2K launches (3K
// with a coupled member), with the ping-pong-only kernels when every member
// uses that store.
int graph_for(lbm_batch_ctx *b, int K, cudaGraphExec_t *out)
{
    const int key = 4 * K + (b->pp ? 2 : 0) + (b->coupled ? 1 : 0);
    for (auto &g : b->graphs)
        if (g.first == key) {
            *out = g.second;
            return LBM_OK;
        }
    cudaGraph_t graph = nullptr;
    int rc = bcuda(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    if (rc != LBM_OK) return rc;
    cudaError_t e1 = cudaMemcpyAsync(b->d_table, b->h_table, b->table_bytes, cudaMemcpyHostToDevice, b->stream);
    cudaError_t e2 = b->ops->batch_launch(b->stream, b->d_table, K, b->grid[0], b->grid[1], b->coupled, b->pp);
    cudaError_t e3 = cudaStreamEndCapture(b->stream, &graph);
    rc = bcuda(b, e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3), "graph capture");
    if (rc != LBM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    cudaGraphExec_t exec = nullptr;
    rc = bcuda(b, cudaGraphInstantiate(&exec, graph, 0), "cudaGraphInstantiate");
    cudaGraphDestroy(graph);
    if (rc != LBM_OK) return rc;
    b->graphs.emplace_back(key, exec);
    *out = exec;
    return LBM_OK;
}

int find_member(const lbm_batch_ctx *b, const lbm_ctx *h)
{
    for (size_t j = 0; j < b->members.size(); ++j)
        if (b->members[j] == h) return (int)j;
    return -1;
}

}  // namespace

extern "C" {

int lbm_batch_create(int lattice, int storage, lbm_batch *out)
{
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    const Ops *ops = ops_for(lattice, storage);
    if (!ops) return LBM_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    lbm_batch_ctx *b = new (std::nothrow) lbm_batch_ctx();
    if (!b) return LBM_ERR_OOM;
    b->lattice = lattice;
    b->storage = storage;
    b->ops = ops;
    cudaGetDevice(&b->device);
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        return LBM_ERR_CUDA;
    }
    b->own_stream = true;
    b->grid[0] = ops->batch_grid(0, 0);
    b->grid[1] = ops->batch_grid(1, 0);
    *out = b;
    return LBM_OK;
}

int lbm_batch_destroy(lbm_batch b)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    cudaStreamSynchronize(b->stream);
    for (lbm_ctx *h : b->members) h->batch = nullptr;
    b->members.clear();
    drop_graphs(b);
    if (b->d_table) cudaFree(b->d_table);
    if (b->h_table) cudaFreeHost(b->h_table);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return LBM_OK;
}

int lbm_batch_set_stream(lbm_batch b, void *stream)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    if (stream) {
        if (b->own_stream) cudaStreamDestroy(b->stream);
        b->own_stream = false;
        b->stream = static_cast<cudaStream_t>(stream);
    } else if (!b->own_stream) {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bfail(b, LBM_ERR_CUDA, "cudaStreamCreateWithFlags");
        b->own_stream = true;
    }
    return LBM_OK;
}

int lbm_batch_set_tuning(lbm_batch b, int chunk, int use_graph)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    if (chunk < 1 || chunk > kBatchMaxChunk || (use_graph != 0 && use_graph != 1))
        return bfail(b, LBM_ERR_INVALID_ARG, "chunk in 1..64, use_graph 0 or 1");
    b->chunk = chunk;
    b->use_graph = use_graph != 0;
    return LBM_OK;
}

int lbm_batch_set_shape(lbm_batch b, int span, int blocks_per_sm)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    if (span < 1 || span > kBatchMaxSpan || blocks_per_sm < 0 || blocks_per_sm > 32)
        return bfail(b, LBM_ERR_INVALID_ARG, "span in 1..16, blocks_per_sm in 0..32");
    cudaStreamSynchronize(b->stream);
    b->span = span;
    if (blocks_per_sm != b->blocks_per_sm) {
        b->blocks_per_sm = blocks_per_sm;
        b->grid[0] = b->ops->batch_grid(0, blocks_per_sm);
        b->grid[1] = b->ops->batch_grid(1, blocks_per_sm);
        drop_graphs(b);   // the captured launches carry the grid
    }
    return LBM_OK;
}

int lbm_batch_add(lbm_batch b, lbm_handle h, int64_t steps)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    if (!h || steps < 0) return bfail(b, LBM_ERR_INVALID_ARG, "NULL handle or steps < 0");
    if (h->batch) return bfail(b, LBM_ERR_INVALID_ARG, "the handle already belongs to a batch");
    if (h->lattice != b->lattice || h->storage != b->storage)
        return bfail(b, LBM_ERR_INVALID_ARG, "the handle's lattice or storage differs from the batch's");
    if (h->device != b->device) return bfail(b, LBM_ERR_INVALID_ARG, "the handle lives on another device");
    if ((unsigned long long)h->Q * (unsigned long long)h->N >= (1ULL << 32))
        return bfail(b, LBM_ERR_UNSUPPORTED, "batch members need Q * sites < 2^32 (32-bit indices)");
    const int rc = ensure_table(b, b->members.size() + 1);
    if (rc != LBM_OK) return rc;
    // the member's earlier work (initialisation, steps) precedes the batch's
    cudaStreamSynchronize(h->stream);
    b->members.push_back(h);
    b->remaining.push_back(steps);
    b->paused.push_back(0);
    h->batch = b;
    return LBM_OK;
}

int lbm_batch_remove(lbm_batch b, lbm_handle h)
{
    if (!b || !h) return LBM_ERR_INVALID_ARG;
    const int j = find_member(b, h);
    if (j < 0) return bfail(b, LBM_ERR_INVALID_ARG, "the handle is not a member of this batch");
    cudaStreamSynchronize(b->stream);
    b->members.erase(b->members.begin() + j);
    b->remaining.erase(b->remaining.begin() + j);
    b->paused.erase(b->paused.begin() + j);
    h->batch = nullptr;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch b, int64_t n, int *finished)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    if (n < 0) return bfail(b, LBM_ERR_INVALID_ARG, "n < 0");
    int rc = LBM_OK;
    const size_t mbytes = b->ops->batch_member_bytes();
    std::vector<int> order, take;
    while (n > 0 && rc == LBM_OK) {
        const int K = (int)std::min<int64_t>(b->chunk, n);
        order.clear();
        take.assign(b->members.size(), 0);
        for (size_t j = 0; j < b->members.size(); ++j) {
            take[j] = b->paused[j] ? 0 : (int)std::min<int64_t>(K, b->remaining[j]);
            if (take[j] > 0) order.push_back((int)j);
        }
        if (order.empty()) break;
        // packed state words (and, with BF16 storage, the deferred odd part
        // of g) of members whose state was (re)loaded or fused-stepped
        for (int j : order) {
            lbm_ctx *h = b->members[j];
            const bool godd = h->storage == LBM_STORE_BF16DEV;
            if (h->fa_valid && (h->g_deferred || !godd)) continue;
            rc = b->ops->split_prepare(h);
            if (rc == LBM_OK) rc = bcuda(b, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize(member)");
            if (rc != LBM_OK) {
                b->err = "packing a member's state failed: " + h->err;
                return rc;
            }
        }
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return take[x] > take[y]; });
        // table: header + members by descending take
        BatchHeader hdr;
        std::memset(&hdr, 0, sizeof hdr);
        hdr.nmem = (long long)order.size();
        hdr.span = b->span;
        char *mem = static_cast<char *>(b->h_table) + batch_header_bytes();
        long long first = 0;
        b->coupled = false;
        b->pp = true;
        for (size_t r = 0; r < order.size(); ++r) {
            const lbm_ctx *h = b->members[order[r]];
            if (h->consts.coupling) b->coupled = true;
            if (h->inplace) b->pp = false;
            b->ops->batch_fill(h, take[order[r]], first, mem + r * mbytes);
            const long long items = b->ops->batch_items(h, b->span);
            for (int k = 0; k < take[order[r]]; ++k) hdr.active[k] += items;
            first += items;
        }
        // launch k covers the members with take > k: a prefix, since sorted
        for (int k = 1; k < K; ++k) hdr.active[k] = std::min(hdr.active[k], hdr.active[k - 1]);
        std::memcpy(b->h_table, &hdr, sizeof hdr);
        if (b->use_graph) {
            cudaGraphExec_t exec = nullptr;
            rc = graph_for(b, K, &exec);
            if (rc == LBM_OK) rc = bcuda(b, cudaGraphLaunch(exec, b->stream), "cudaGraphLaunch");
        } else {
            rc = bcuda(b, cudaMemcpyAsync(b->d_table, b->h_table, b->table_bytes, cudaMemcpyHostToDevice, b->stream),
                       "H2D batch table");
            if (rc == LBM_OK)
                rc = bcuda(b, b->ops->batch_launch(b->stream, b->d_table, K, b->grid[0], b->grid[1], b->coupled,
                                                   b->pp),
                           "batch launch");
        }
        // the pinned table is rewritten for the next chunk: wait for this one
        if (rc == LBM_OK) rc = bcuda(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize(batch)");
        if (rc != LBM_OK) break;
        b->launches += (b->coupled ? 3LL : 2LL) * K;
        for (int j : order) {
            lbm_ctx *h = b->members[j];
            h->steps += take[j];
            if (take[j] & 1) h->cur = 1 - h->cur;
            if (h->storage != LBM_STORE_F64) h->soa_valid = false;   // the state is in fa[cur]
            if (h->storage == LBM_STORE_BF16DEV) h->g_deferred = true;
            b->remaining[j] -= take[j];
        }
        n -= K;
    }
    if (finished) {
        int f = 0;
        for (int64_t r : b->remaining) f += (r == 0);
        *finished = f;
    }
    return rc;
}

int lbm_batch_pause(lbm_batch b, lbm_handle h, int32_t paused)
{
    if (!b || !h) return LBM_ERR_INVALID_ARG;
    if (paused != 0 && paused != 1) return bfail(b, LBM_ERR_INVALID_ARG, "paused is 0 or 1");
    const int j = find_member(b, h);
    if (j < 0) return bfail(b, LBM_ERR_INVALID_ARG, "the handle is not a member of this batch");
    b->paused[j] = (char)paused;
    return LBM_OK;
}

int lbm_batch_remaining(lbm_batch b, lbm_handle h, int64_t *steps_left)
{
    if (!b || !h || !steps_left) return LBM_ERR_INVALID_ARG;
    const int j = find_member(b, h);
    if (j < 0) return bfail(b, LBM_ERR_INVALID_ARG, "the handle is not a member of this batch");
    *steps_left = b->remaining[j];
    return LBM_OK;
}

int lbm_batch_info(lbm_batch b, int *members, int64_t *launches)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    if (members) *members = (int)b->members.size();
    if (launches) *launches = b->launches;
    return LBM_OK;
}

const char *lbm_batch_last_error(lbm_batch b)
{
    static const char *none = "invalid batch";
    return b ? b->err.c_str() : none;
}

// ---------------------------------------------------------------------------

int lbm_batch_autotune(lbm_batch b, int trial_steps, int *chunk, int *span, int *blocks_per_sm, double *ms_per_step)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    if (trial_steps < 1 || trial_steps > 1000) return bfail(b, LBM_ERR_INVALID_ARG, "trial_steps in 1..1000");
    if (b->members.empty()) return bfail(b, LBM_ERR_INVALID_ARG, "the batch has no members");
    // every member's state and budget, restored after the trials
    std::vector<std::vector<char>> saved(b->members.size());
    std::vector<int64_t> budget = b->remaining;
    const std::vector<char> paused = b->paused;   // every member steps in the trials
    std::fill(b->paused.begin(), b->paused.end(), 0);
    int rc = LBM_OK;
    for (size_t j = 0; j < b->members.size() && rc == LBM_OK; ++j) {
        size_t bytes = 0;
        rc = lbm_state_bytes(b->members[j], &bytes);
        if (rc == LBM_OK) {
            saved[j].resize(bytes);
            rc = lbm_save_state(b->members[j], saved[j].data(), bytes);
        }
    }
    if (rc != LBM_OK) {
        b->paused = paused;
        return bfail(b, rc, "saving a member's state failed");
    }
    const int chunk0 = b->chunk, span0 = b->span, bps0 = b->blocks_per_sm;
    int occ = 0;
    {
        int sms = 1;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
        occ = b->ops->batch_grid(0, 0) / (sms > 0 ? sms : 1);
    }
    struct Cand {
        int chunk, span, bps;
    };
    std::vector<Cand> cands;
    for (int K : {8, 16, 32})
        for (int sp : {1, 2, 4, 8})
            for (int bps : {0, occ > 2 ? occ - 1 : 0}) {
                if (bps != 0 && bps == occ) continue;
                bool dup = false;
                for (const Cand &c : cands) dup = dup || (c.chunk == K && c.span == sp && c.bps == bps);
                if (!dup) cands.push_back({K, sp, bps});
            }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e300;
    Cand pick{chunk0, span0, bps0};
    for (const Cand &c : cands) {
        rc = lbm_batch_set_shape(b, c.span, c.bps);
        if (rc == LBM_OK) rc = lbm_batch_set_tuning(b, c.chunk, b->use_graph ? 1 : 0);
        for (size_t j = 0; j < b->members.size(); ++j) b->remaining[j] = 1 << 30;
        if (rc == LBM_OK) rc = lbm_batch_step(b, c.chunk, nullptr);   // warm-up: graph capture
        if (rc != LBM_OK) break;
        cudaEventRecord(e0, b->stream);
        const int steps = (trial_steps + c.chunk - 1) / c.chunk * c.chunk;
        rc = lbm_batch_step(b, steps, nullptr);
        cudaEventRecord(e1, b->stream);
        if (rc != LBM_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = bcuda(b, cudaGetLastError(), "batch autotune timing");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = ms / steps;
        if (per < best) {
            best = per;
            pick = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the members continue from their saved states, with their budgets
    int rc_restore = LBM_OK;
    for (size_t j = 0; j < b->members.size(); ++j) {
        const int r = lbm_load_state(b->members[j], saved[j].data(), saved[j].size());
        if (r != LBM_OK && rc_restore == LBM_OK) rc_restore = r;
    }
    b->remaining = budget;
    b->paused = paused;
    if (rc != LBM_OK) {
        lbm_batch_set_shape(b, span0, bps0);
        lbm_batch_set_tuning(b, chunk0, b->use_graph ? 1 : 0);
        return rc;
    }
    if (rc_restore != LBM_OK) return bfail(b, rc_restore, "restoring a member's state failed");
    rc = lbm_batch_set_shape(b, pick.span, pick.bps);
    if (rc == LBM_OK) rc = lbm_batch_set_tuning(b, pick.chunk, b->use_graph ? 1 : 0);
    if (rc != LBM_OK) return rc;
    if (chunk) *chunk = pick.chunk;
    if (span) *span = pick.span;
    if (blocks_per_sm) *blocks_per_sm = pick.bps;
    if (ms_per_step) *ms_per_step = best;
    return LBM_OK;
}

int lbm_autotune(lbm_handle h, int trial_steps, int *variant, int *zchunk, double *ms_per_step)
{
    if (!h) return LBM_ERR_INVALID_ARG;
    if (trial_steps < 1 || trial_steps > 1000) {
        h->err = "trial_steps in 1..1000";
        return LBM_ERR_INVALID_ARG;
    }
    if (h->batch) {
        h->err = "the handle is stepped by its batch";
        return LBM_ERR_INVALID_ARG;
    }
    struct Cand {
        int variant, zchunk, rows, staged;
    };
    std::vector<Cand> cands;
    cands.push_back({3, 0, 0, -1});
    if (h->ops->persist_ok(h)) cands.push_back({4, 0, 0, -1});
    if (!h->inplace) {
        cands.push_back({1, 0, 0, -1});
        if (h->ops->has_v2() && h->D == 3)
            for (int zc : {0, 4, 8, 16, 32, 64})
                if (zc <= h->nz) cands.push_back({2, zc, 0, -1});
        if (!h->consts.coupling)
            for (int rows : {4, 8, 16})
                if (h->ops->cluster_ok(h, rows))
                    for (int st : {0, 1})
                        for (int zc : {0, 64})
                            if (zc <= h->nz) cands.push_back({5, zc, rows, st});
    }
    const int v0 = h->variant, z0 = h->zchunk, r0 = h->cluster_rows, s0 = h->cluster_stage;
    if (cands.size() == 1) {
        h->variant = cands[0].variant;
        if (variant) *variant = cands[0].variant;
        if (zchunk) *zchunk = 0;
        if (ms_per_step) *ms_per_step = 0.0;
        return LBM_OK;
    }
    size_t bytes = 0;
    lbm_state_bytes(h, &bytes);
    std::vector<char> saved(bytes);
    int rc = lbm_save_state(h, saved.data(), bytes);
    if (rc != LBM_OK) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e300;
    Cand pick = cands[0];
    for (const Cand &c : cands) {
        if (c.variant == 5) {
            rc = lbm_set_cluster(h, c.rows, c.staged);
            if (rc == LBM_ERR_UNSUPPORTED) {   // e.g. clusters of 16 not allowed on the device
                rc = LBM_OK;
                continue;
            }
            if (rc != LBM_OK) break;
        }
        rc = lbm_set_tuning(h, c.variant, c.zchunk);
        if (rc != LBM_OK) break;
        rc = h->ops->step(h, 1);   // warm-up (and first-use attributes)
        if (rc != LBM_OK) break;
        cudaEventRecord(e0, h->stream);
        rc = h->ops->step(h, trial_steps);
        cudaEventRecord(e1, h->stream);
        if (rc != LBM_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = cuda_fail(h, cudaGetLastError(), "autotune timing");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = ms / trial_steps;
        if (per < best) {
            best = per;
            pick = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const int rc_restore = lbm_load_state(h, saved.data(), bytes);
    if (rc != LBM_OK) {
        h->variant = v0;
        h->zchunk = z0;
        h->cluster_rows = r0;
        h->cluster_stage = s0;
        return rc;
    }
    if (rc_restore != LBM_OK) return rc_restore;
    if (pick.variant == 5) rc = lbm_set_cluster(h, pick.rows, pick.staged);
    if (rc == LBM_OK) rc = lbm_set_tuning(h, pick.variant, pick.zchunk);
    if (rc != LBM_OK) return rc;
    if (variant) *variant = pick.variant;
    if (zchunk) *zchunk = pick.zchunk;
    if (ms_per_step) *ms_per_step = best;
    return LBM_OK;
}

}  // extern "C"
