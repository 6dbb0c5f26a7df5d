// Batches of independent registration problems (many pairs of uneven
// sizes): the host-side plan of the persistent batch kernel, its autotuner
// and the C ABI. Declarations and contracts: include/airgb.h.
//
// The plan lays out one workspace: the queue and per-problem counters, an
// error word, the problem descriptors, the work-item list and each problem's
// partial sums. One iteration is a memset of the counters and one launch of
// k_batch (kernels_fused.cu); both can be captured in a CUDA graph.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "airgb.h"
#include "checks.h"
#include "launch.h"

using namespace airgb;

namespace {

size_t a256(size_t b) { return (b + 255) / 256 * 256; }

constexpr int kPolicies = 4;
constexpr int kMaxTiles = 4;

// A problem's plan for every brick tile of the batch kernel (the workspace
// holds the largest tile's partials, so a tile can change after binding).
struct ProbPlan {
    Grid g;
    Lattice L;
    double lambda;
    int gt[3], ngram, nmom;
    int gb[kMaxTiles][3], npart[kMaxTiles], nbricks[kMaxTiles], nchunks[kMaxTiles];
    size_t bpart, mpart, rpart, gR;  // workspace offsets
    double work;                     // voxels, for ordering
};

}  // namespace

struct al_batch {
    int delta = 0;
    std::vector<ProbPlan> prob;
    size_t off_counters = 0, off_err = 0, off_desc = 0, off_items = 0, total = 0;
    int ntiles = 1;
    int tile = 0;                       // brick tile of the batch kernel in use
    int nitems = 0;                     // items of one iteration with that tile
    int policy = 1;
    int blocks = 0;
    std::vector<BatchProblem> desc;     // bound descriptors (host copy)
    int extra_wait = 0;
    long long spin_limit = 20000000;  // about 3 s of polling
    char *ws = nullptr;               // bound workspace
};

namespace {

// Work items in the order of a policy. Every phase A item (bricks, Gram
// tiles) precedes every phase B item (control chunks); the kernel's waits
// rely on it.
//  0: problems in the given order, each problem's bricks then its tiles;
//  1: largest problem first (by voxels), same grouping;
//  2: round-robin over the problems, one item at a time;
//  3: every Gram tile first (largest problem first), then the bricks.
std::vector<BatchItem> make_items(const al_batch &b, int policy)
{
    const int n = (int)b.prob.size(), t = b.tile;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i)
        order[i] = i;
    if (policy == 1 || policy == 3)
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int c) { return b.prob[a].work > b.prob[c].work; });
    std::vector<BatchItem> v;
    if (policy == 2) {
        std::vector<int> nb(n, 0), ng(n, 0);
        bool more = true;
        while (more) {
            more = false;
            for (int i = 0; i < n; ++i) {
                const ProbPlan &p = b.prob[i];
                if (nb[i] < p.nbricks[t]) {
                    v.push_back({i, BATCH_BRICK, nb[i]++, 0});
                    more = true;
                } else if (ng[i] < p.ngram) {
                    v.push_back({i, BATCH_GRAM, ng[i]++, 0});
                    more = true;
                }
            }
        }
    } else if (policy == 3) {
        for (int i : order)
            for (int t = 0; t < b.prob[i].ngram; ++t)
                v.push_back({i, BATCH_GRAM, t, 0});
        for (int i : order)
            for (int k = 0; k < b.prob[i].nbricks[t]; ++k)
                v.push_back({i, BATCH_BRICK, k, 0});
    } else {
        for (int i : order) {
            for (int k = 0; k < b.prob[i].nbricks[t]; ++k)
                v.push_back({i, BATCH_BRICK, k, 0});
            for (int t = 0; t < b.prob[i].ngram; ++t)
                v.push_back({i, BATCH_GRAM, t, 0});
        }
    }
    for (int i : order)
        for (int k = 0; k < b.prob[i].nchunks[t]; ++k)
            v.push_back({i, BATCH_CTRL, k, 0});
    return v;
}

int count_items(const al_batch &b, int t)
{
    int n = 0;
    for (const ProbPlan &p : b.prob)
        n += p.nbricks[t] + p.ngram + p.nchunks[t];
    return n;
}

// Select brick tile t: the descriptors' brick geometry, the launch size and
// the work items (in the current order) follow it.
al_status use_tile(al_batch &b, int t)
{
    const int occ = batch_blocks_per_sm(b.delta, t);
    if (occ < 1)
        return AL_ERR_CUDA;
    for (size_t i = 0; i < b.prob.size(); ++i) {
        const ProbPlan &p = b.prob[i];
        BatchProblem &q = b.desc[i];
        q.gbx = p.gb[t][0];
        q.gby = p.gb[t][1];
        q.gbz = p.gb[t][2];
        q.nbricks = p.nbricks[t];
        q.nA = p.nbricks[t] + p.ngram;
        q.nchunks = p.nchunks[t];
    }
    if (cudaMemcpy(b.ws + b.off_desc, b.desc.data(), sizeof(BatchProblem) * b.desc.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return AL_ERR_CUDA;
    b.tile = t;
    b.nitems = count_items(b, t);
    b.blocks = occ * device_sms();  // persistent: resident blocks of every SM
    const std::vector<BatchItem> v = make_items(b, b.policy);
    if (cudaMemcpy(b.ws + b.off_items, v.data(), v.size() * sizeof(BatchItem),
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return AL_ERR_CUDA;
    return AL_OK;
}

al_status upload_items(al_batch &b, int policy)
{
    const std::vector<BatchItem> v = make_items(b, policy);
    if ((int)v.size() != b.nitems)
        return AL_ERR_INVALID_ARG;
    if (cudaMemcpy(b.ws + b.off_items, v.data(), v.size() * sizeof(BatchItem),
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return AL_ERR_CUDA;
    b.policy = policy;
    return AL_OK;
}

al_status launch_step(const al_batch &b, const BatchStep &st, cudaStream_t s)
{
    int *counters = (int *)(b.ws + b.off_counters);
    if (cudaMemsetAsync(counters, 0, sizeof(int) * (1 + b.prob.size()), s) != cudaSuccess)
        return AL_ERR_CUDA;
    const int blocks = b.blocks > 0 ? b.blocks : device_sms();
    return launched(launch_batch(b.delta, b.tile, blocks,
                                 (const BatchProblem *)(b.ws + b.off_desc),
                                 (const BatchItem *)(b.ws + b.off_items), b.nitems, counters, st,
                                 s));
}

BatchStep step_args(const al_batch &b, const al_adam_params &p, int64_t t, int record, int update)
{
    BatchStep st{};
    st.beta1 = p.beta1;
    st.beta2 = p.beta2;
    st.lr = (float)p.lr;
    st.eps = (float)p.eps;
    st.t = t;
    st.record = record;
    st.update = update;
    st.extra_wait = b.extra_wait;
    st.spin_limit = b.spin_limit;
    st.err = (int *)(b.ws + b.off_err);
    return st;
}

bool adam_ok(const al_adam_params *p)
{
    return p && p->lr >= 0.0 && isfinite(p->lr) && p->beta1 >= 0.0 && p->beta1 < 1.0 &&
           p->beta2 >= 0.0 && p->beta2 < 1.0 && p->eps > 0.0 && isfinite(p->eps);
}

}  // namespace

extern "C" {

al_status al_batch_create(const al_problem *problems, int32_t count, al_batch **out)
{
    if (!problems || !out || count < 1)
        return AL_ERR_INVALID_ARG;
    *out = nullptr;
    al_batch *b = new (std::nothrow) al_batch();
    if (!b)
        return AL_ERR_INVALID_ARG;
    size_t off = 0;
    b->off_counters = off;
    off += a256(sizeof(int) * (1 + (size_t)count));
    b->off_err = off;
    off += 256;
    b->off_desc = off;
    off += a256(sizeof(BatchProblem) * (size_t)count);
    int nitems = 0;
    for (int i = 0; i < count; ++i) {
        const al_problem &pr = problems[i];
        ProbPlan p{};
        al_status st = check_bspline(&pr.bs, &p.g, &p.L);
        if (st == AL_OK)
            st = check_sim(&pr.sim, p.g.ndim);
        if (st == AL_OK && !isfinite(pr.lambda))
            st = AL_ERR_INVALID_ARG;
        if (st == AL_OK && (pr.sim.kind != AL_SIM_MSE || batch_threads(pr.bs.spacing, 0) == 0 ||
                            (i > 0 && pr.bs.spacing != problems[0].bs.spacing)))
            st = AL_ERR_UNSUPPORTED;  // MSE, one spacing in {4, 6, 8}
        if (st != AL_OK) {
            delete b;
            return st;
        }
        p.lambda = pr.lambda;
        b->ntiles = batch_tiles() < kMaxTiles ? batch_tiles() : kMaxTiles;
        for (int t = 0; t < b->ntiles; ++t) {
            batch_geometry(p.g, p.L, t, p.gb[t], p.gt, &p.npart[t], &p.nmom);
            p.nbricks[t] = p.gb[t][0] * p.gb[t][1] * p.gb[t][2];
            const int threads = batch_threads(pr.bs.spacing, t);
            p.nchunks[t] = (p.L.nc + threads - 1) / threads;
        }
        p.ngram = p.g.ndim * p.gt[0] * p.gt[1] * p.gt[2];
        p.work = (double)p.g.nv;
        b->prob.push_back(p);
    }
    b->delta = problems[0].bs.spacing;
    for (int t = 0; t < b->ntiles; ++t)
        nitems = std::max(nitems, count_items(*b, t));
    b->nitems = count_items(*b, 0);
    b->off_items = off;
    off += a256(sizeof(BatchItem) * (size_t)nitems);
    for (ProbPlan &p : b->prob) {
        size_t part = 0, mom = 0;  // the largest tile's partials
        for (int t = 0; t < b->ntiles; ++t) {
            part = std::max(part, (size_t)p.nbricks[t] * p.npart[t]);
            mom = std::max(mom, (size_t)p.nbricks[t] * p.nmom);
        }
        p.bpart = off;
        off += a256(part * sizeof(float));
        p.mpart = off;
        off += a256(mom * sizeof(double));
        p.rpart = off;
        off += a256((size_t)p.ngram * sizeof(double));
        p.gR = off;
        off += a256((size_t)p.g.ndim * p.L.nc * sizeof(float));
    }
    b->total = off;
    *out = b;
    return AL_OK;
}

void al_batch_destroy(al_batch *b) { delete b; }

size_t al_batch_workspace_bytes(const al_batch *b) { return b ? b->total : 0; }

int32_t al_batch_items(const al_batch *b, int32_t *per_kind)
{
    if (!b)
        return 0;
    if (per_kind) {
        per_kind[0] = per_kind[1] = per_kind[2] = 0;
        for (const ProbPlan &p : b->prob) {
            per_kind[0] += p.nbricks[b->tile];
            per_kind[1] += p.ngram;
            per_kind[2] += p.nchunks[b->tile];
        }
    }
    return b->nitems;
}

al_status al_batch_bind(al_batch *b, const float *const *fixed, const float *const *moving,
                        float *const *ctrl, float *const *adam_m, float *const *adam_v,
                        double *const *values, void *workspace, size_t workspace_bytes)
{
    if (!b || !fixed || !moving || !ctrl || !adam_m || !adam_v)
        return AL_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < b->total)
        return AL_ERR_WORKSPACE;
    if (!aligned16(workspace))
        return AL_ERR_ALIGN;
    const int n = (int)b->prob.size();
    for (int i = 0; i < n; ++i) {
        if (!fixed[i] || !moving[i] || !ctrl[i] || !adam_m[i] || !adam_v[i])
            return AL_ERR_INVALID_ARG;
        if (!aligned16(fixed[i]) || !aligned16(moving[i]) || !aligned16(ctrl[i]) ||
            !aligned16(adam_m[i]) || !aligned16(adam_v[i]) || (values && values[i] &&
                                                               !aligned16(values[i])))
            return AL_ERR_ALIGN;
    }
    char *ws = (char *)workspace;
    std::vector<BatchProblem> d(n);
    for (int i = 0; i < n; ++i) {
        const ProbPlan &p = b->prob[i];
        BatchProblem &q = d[i];
        memset(&q, 0, sizeof(q));
        q.g = p.g;
        q.L = p.L;
        q.F = fixed[i];
        q.M = moving[i];
        q.c = ctrl[i];
        q.m = adam_m[i];
        q.v = adam_v[i];
        q.values = values ? values[i] : nullptr;
        q.bpart = (float *)(ws + p.bpart);
        q.mpart = (double *)(ws + p.mpart);
        q.rpart = (double *)(ws + p.rpart);
        q.gR = (float *)(ws + p.gR);
        const int N[3] = {p.g.X, p.g.Y, p.g.Z};
        for (int k = 0; k < 3; ++k)
            q.h[k] = k < p.g.ndim ? (float)((N[k] - 1) / 2.0) : 0.0f;
        q.gscale = (float)(2.0 / (double)p.g.nv);
        q.lambda = p.lambda;
        q.gtx = p.gt[0];
        q.gty = p.gt[1];
        q.gtz = p.gt[2];
        q.ngram = p.ngram;  // brick geometry: use_tile
    }
    if (cudaMemset(ws + b->off_err, 0, sizeof(int)) != cudaSuccess)
        return AL_ERR_CUDA;
    b->ws = ws;
    b->desc = d;
    return use_tile(*b, b->tile);
}

al_status al_batch_step(const al_batch *b, const al_adam_params *p, int64_t step, int32_t record,
                        al_stream stream)
{
    if (!b || !adam_ok(p) || step < 1)
        return AL_ERR_INVALID_ARG;
    if (!b->ws)
        return AL_ERR_WORKSPACE;
    return launch_step(*b, step_args(*b, *p, step, record, 1), (cudaStream_t)stream);
}

al_status al_batch_tune(al_batch *b, const al_adam_params *p, int32_t iterations, double *ms,
                        int32_t *chosen_tile, int32_t *chosen_policy, al_stream stream)
{
    if (!b || !adam_ok(p) || iterations < 1)
        return AL_ERR_INVALID_ARG;
    if (!b->ws)
        return AL_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return AL_ERR_CUDA;
    const BatchStep st = step_args(*b, *p, 1, -1, 0);  // gradients only: state unchanged
    double best = 1e300;
    int best_policy = b->policy, best_tile = b->tile;
    al_status rc = AL_OK;
    for (int cfg = 0; cfg < b->ntiles * kPolicies && rc == AL_OK; ++cfg) {
        const int tile = cfg / kPolicies, pol = cfg % kPolicies;
        if (cudaStreamSynchronize(s) != cudaSuccess) {  // the bound descriptors are rewritten
            rc = AL_ERR_CUDA;
            break;
        }
        b->policy = pol;
        if ((rc = use_tile(*b, tile)) != AL_OK)
            break;
        for (int w = 0; w < 2 && rc == AL_OK; ++w)
            rc = launch_step(*b, st, s);
        if (rc != AL_OK || cudaEventRecord(e0, s) != cudaSuccess) {
            rc = rc == AL_OK ? AL_ERR_CUDA : rc;
            break;
        }
        for (int it = 0; it < iterations && rc == AL_OK; ++it)
            rc = launch_step(*b, st, s);
        float t = 0.0f;
        if (rc != AL_OK || cudaEventRecord(e1, s) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
            rc = rc == AL_OK ? AL_ERR_CUDA : rc;
            break;
        }
        const double per = (double)t / iterations;
        if (ms)
            ms[cfg] = per;
        if (per < best) {
            best = per;
            best_policy = pol;
            best_tile = tile;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != AL_OK)
        return rc;
    if (chosen_tile)
        *chosen_tile = best_tile;
    if (chosen_policy)
        *chosen_policy = best_policy;
    b->policy = best_policy;
    return use_tile(*b, best_tile);
}

al_status al_batch_set_tile(al_batch *b, int32_t tile)
{
    if (!b || tile < 0 || tile >= b->ntiles)
        return AL_ERR_INVALID_ARG;
    if (!b->ws) {
        b->tile = tile;
        b->nitems = count_items(*b, tile);
        return AL_OK;
    }
    return use_tile(*b, tile);
}

int32_t al_batch_tiles(const al_batch *b, int32_t *cells)
{
    if (!b)
        return 0;
    if (cells)
        for (int t = 0; t < b->ntiles; ++t)
            batch_tile_cells(b->delta, t, &cells[2 * t], &cells[2 * t + 1]);
    return b->ntiles;
}

al_status al_batch_set_policy(al_batch *b, int32_t policy)
{
    if (!b || policy < 0 || policy >= kPolicies)
        return AL_ERR_INVALID_ARG;
    if (!b->ws) {
        b->policy = policy;
        return AL_OK;
    }
    return upload_items(*b, policy);
}

al_status al_batch_set_wait(al_batch *b, int32_t extra_items, int64_t max_polls)
{
    if (!b || extra_items < 0 || max_polls < 1)
        return AL_ERR_INVALID_ARG;
    b->extra_wait = extra_items;
    b->spin_limit = max_polls;
    return AL_OK;
}

al_status al_batch_status(const al_batch *b, al_stream stream)
{
    if (!b)
        return AL_ERR_INVALID_ARG;
    if (!b->ws)
        return AL_ERR_WORKSPACE;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return AL_ERR_CUDA;
    int h = 0;
    if (cudaMemcpy(&h, b->ws + b->off_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return AL_ERR_CUDA;
    if (h != 0 && cudaMemset(b->ws + b->off_err, 0, sizeof(int)) != cudaSuccess)
        return AL_ERR_CUDA;
    return (al_status)h;
}

}  // extern "C"
