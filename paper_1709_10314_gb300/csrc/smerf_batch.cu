// smerf_batch.cu -- batched sampling: many requests (plans of different grids, spectra and
// precisions) in few launches.  Requests with FP32 recursion run in two persistent phases per
// table precision: one anchor launch over every request's anchor items, then one launch of
// persistent CTAs that pull segment items of every shape (p, n_phi, launch configuration) from
// a device queue, largest first.  Requests with FP64 recursion or p = 3 form groups of one
// kernel shape that run as one anchor launch and one segment launch each.  Per-request
// parameters (tables, seed, output, scratch) are read from a descriptor array in device
// memory.  The work lists and the scratch are built once per batch, so a launch (descriptor
// copy, queue reset, kernels) can be captured into a CUDA graph and replayed with new seeds and
// outputs.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "smerf_internal.cuh"

using smerf::SampleParams;

namespace {

enum Kind { kFF = 0, kFD = 1, kDD = 2, kDF = 3 };

int kind_of(const smerf_plan* pl) { return pl->recur64 ? (pl->tab64 ? kDD : kDF) : (pl->tab64 ? kFD : kFF); }

int fill_params(int kind, const smerf_plan* pl, uint64_t seed, int n, void* out, void* scratch, SampleParams* P,
                int* batchable, int* rmax)
{
    switch (kind) {
        case kFF: return smerf_fill_params_ff(pl, seed, n, out, scratch, P, batchable, rmax);
        case kFD: return smerf_fill_params_fd(pl, seed, n, out, scratch, P, batchable, rmax);
        case kDD: return smerf_fill_params_dd(pl, seed, n, out, scratch, P, batchable, rmax);
        default: return smerf_fill_params_df(pl, seed, n, out, scratch, P, batchable, rmax);
    }
}

// FP32-recursion groups with p <= 2 run in the persistent launch (p = 3, whose units hold 12
// state values, keeps a launch pair per group so that the persistent kernel's registers stay
// sized for p <= 2)
bool queued(int kind, int p) { return (kind == kFF || kind == kFD) && p <= 2; }

// A queued kind's work: its items (every anchor item, then every segment item, each list
// largest request first), the persistent launch's shared memory and CTAs, and its control
// words (queue head, status, one anchor counter per request of the batch).
struct Queue {
    int kind;
    int4* d_items = nullptr;   // anchor items (blocks of kQueueThreads units), then segment items
    int n_items = 0;
    int n_anc = 0;
    int4* d_anc128 = nullptr;  // the anchor items in blocks of 128 units (the anchor launch)
    int n_anc128 = 0;
    size_t smem = 0;
    int ctas = 0;
    int* d_ctl = nullptr;
};

int launch_queue(const Queue& q, const SampleParams* d, int n_req, int single, int fail_waits, cudaStream_t st)
{
    return q.kind == kFF ? smerf_launch_queue_ff(d, q.d_items, q.n_items, q.n_anc, q.d_anc128, q.n_anc128, q.d_ctl,
                                                 n_req, single, fail_waits, q.smem, q.ctas, st)
                         : smerf_launch_queue_fd(d, q.d_items, q.n_items, q.n_anc, q.d_anc128, q.n_anc128, q.d_ctl,
                                                 n_req, single, fail_waits, q.smem, q.ctas, st);
}

int queue_ctas(int kind, size_t smem)
{
    return kind == kFF ? smerf_queue_ctas_ff(smem) : smerf_queue_ctas_fd(smem);
}

int launch_group(int kind, const smerf_plan* rep, const SampleParams* d, const int4* a, int na, const int4* s, int ns,
                 cudaStream_t st)
{
    switch (kind) {
        case kFF: return smerf_launch_group_ff(rep, d, a, na, s, ns, st);
        case kFD: return smerf_launch_group_fd(rep, d, a, na, s, ns, st);
        case kDD: return smerf_launch_group_dd(rep, d, a, na, s, ns, st);
        default: return smerf_launch_group_df(rep, d, a, na, s, ns, st);
    }
}

struct Group {
    int kind;
    const smerf_plan* rep;
    int4* d_anc = nullptr;
    int n_anc = 0;
    int4* d_seg = nullptr;
    int n_seg = 0;
};

}  // namespace

struct smerf_batch {
    int n_req = 0;
    int dev = 0;
    std::vector<const smerf_plan*> plans;
    std::vector<int> counts;
    std::vector<size_t> offs;
    std::vector<int> singles;  // requests whose shape has no batched kernel (launched one by one)
    std::vector<Group> groups;   // kernel shapes (FP64 recursion: launched per group)
    std::vector<Queue> queues;   // FP32 recursion: the persistent work per table precision
    int single = 0;              // 1: one persistent launch per queue; 0: anchor launch + persistent launch
    int fail_waits = 0;          // test hook: the next single launch's anchor waits cannot be met
    void* scratch = nullptr;
    SampleParams* h_descs = nullptr;  // pinned staging
    SampleParams* d_descs = nullptr;
    std::vector<uint64_t> seeds;
    std::vector<void*> outs;
};

static void batch_free(smerf_batch* b)
{
    if (!b) return;
    for (auto& g : b->groups) {
        cudaFree(g.d_anc);
        cudaFree(g.d_seg);
    }
    for (auto& q : b->queues) {
        cudaFree(q.d_items);
        cudaFree(q.d_anc128);
        cudaFree(q.d_ctl);
    }
    cudaFree(b->scratch);
    cudaFree(b->d_descs);
    cudaFreeHost(b->h_descs);
    delete b;
}

extern "C" {

int smerf_batch_create(const smerf_plan* const* plans, const int* n_samples, int n_req, smerf_batch** out)
{
    if (!out) return SMERF_EINVAL;
    *out = nullptr;
    if (n_req < 0 || (n_req > 0 && (!plans || !n_samples))) return SMERF_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SMERF_ECUDA;
    for (int i = 0; i < n_req; ++i)
        if (!plans[i] || n_samples[i] < 0 || n_samples[i] > 65535 || plans[i]->dev != dev) return SMERF_EINVAL;
    smerf_batch* b = new (std::nothrow) smerf_batch;
    if (!b) return SMERF_ENOMEM;
    b->n_req = n_req;
    b->dev = dev;
    b->plans.assign(plans, plans + n_req);
    b->counts.assign(n_samples, n_samples + n_req);
    b->seeds.assign(n_req, 0);
    b->outs.assign(n_req, nullptr);
    size_t total = 0;
    for (int i = 0; i < n_req; ++i) {
        b->offs.push_back(total);
        total += (smerf_scratch_bytes(plans[i], n_samples[i]) + 255) & ~(size_t)255;
    }
    int rc = SMERF_OK;
    if (total && smerf::dev_malloc((void**)&b->scratch, total) != cudaSuccess) rc = SMERF_ENOMEM;
    if (rc == SMERF_OK && n_req) {
        if (smerf::host_malloc((void**)&b->h_descs, sizeof(SampleParams) * n_req) != cudaSuccess ||
            smerf::dev_malloc((void**)&b->d_descs, sizeof(SampleParams) * n_req) != cudaSuccess)
            rc = SMERF_ENOMEM;
    }
    // group by kernel shape; build the work lists
    // requests share a group when their kernels and launch configurations coincide: same
    // precision pair, p, n_phi, anchoring and tuned launch parameters (if any)
    std::map<std::tuple<int, int, int, int, int, int, int, int, int>, int> gidx;
    std::vector<std::vector<int4>> anc, seg;
    for (int i = 0; rc == SMERF_OK && i < n_req; ++i) {
        const smerf_plan* pl = plans[i];
        const int n = n_samples[i];
        int batchable = 0, rmax = 1;
        const int kind = kind_of(pl);
        rc = fill_params(kind, pl, 0, n, nullptr, (char*)b->scratch + b->offs[i], &b->h_descs[i], &batchable, &rmax);
        if (rc != SMERF_OK || n == 0) continue;
        // ring-dependent longitudes: the batched kernels write whole equiangular rings only, so
        // such a request is launched as a single call would launch it
        if (!batchable || pl->rings_total) {
            b->singles.push_back(i);
            continue;
        }
        const bool tuned = pl->tune.valid != 0;
        const auto key = std::make_tuple(kind, pl->p, pl->n_phi, pl->H > 0 ? 1 : 0, tuned ? pl->tune.upt : 0,
                                         tuned ? pl->tune.rmax : 0, tuned ? pl->tune.np : 0, tuned ? pl->tune.nf : 0,
                                         tuned ? pl->tune.minb : 0);
        auto it = gidx.find(key);
        int g;
        if (it == gidx.end()) {
            g = (int)b->groups.size();
            gidx[key] = g;
            Group gr;
            gr.kind = kind;
            gr.rep = pl;
            b->groups.push_back(gr);
            anc.emplace_back();
            seg.emplace_back();
        } else {
            g = it->second;
        }
        const int n_units = pl->n_slots / smerf::unit_slots(pl->p);
        for (int c = 0; c < 2; ++c)
            for (int r = 0; r < n; ++r)
                for (int ub = 0; ub < (n_units + 127) / 128; ++ub) anc[g].push_back(make_int4(i, ub, r, c));
        for (int sgi = 0; sgi < pl->n_segments; ++sgi)
            for (int gr = 0; gr < (n + rmax - 1) / rmax; ++gr) seg[g].push_back(make_int4(i, sgi, gr, 0));
    }
    for (size_t g = 0; rc == SMERF_OK && g < b->groups.size(); ++g) {
        Group& gr = b->groups[g];
        gr.n_anc = (int)anc[g].size();
        gr.n_seg = (int)seg[g].size();
        if (queued(gr.kind, gr.rep->p)) continue;  // its items go to the persistent queue below
        if (smerf::dev_malloc((void**)&gr.d_anc, sizeof(int4) * gr.n_anc) != cudaSuccess ||
            smerf::dev_malloc((void**)&gr.d_seg, sizeof(int4) * gr.n_seg) != cudaSuccess) {
            rc = SMERF_ENOMEM;
            break;
        }
        if (cudaMemcpy(gr.d_anc, anc[g].data(), sizeof(int4) * gr.n_anc, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(gr.d_seg, seg[g].data(), sizeof(int4) * gr.n_seg, cudaMemcpyHostToDevice) != cudaSuccess)
            rc = SMERF_ECUDA;
    }
    // the FP32-recursion requests merged into one queue per table precision; each runs with the
    // queue's build for its size (smerf::queue_build), its descriptor's producer count set to it
    for (int kind : {(int)kFF, (int)kFD}) {
        if (rc != SMERF_OK) break;
        std::vector<std::pair<double, int4>> qa, qa128, qs;  // (request cost or item cost, item)
        size_t smem = 0;
        for (size_t g = 0; g < b->groups.size() && rc == SMERF_OK; ++g) {
            if (b->groups[g].kind != kind || !queued(kind, b->groups[g].rep->p)) continue;
            int last = -1;
            for (const int4& it : seg[g]) {
                const int i = it.x;
                if (i == last) continue;  // the request's items are made below, once
                last = i;
                const smerf_plan* pl = plans[i];
                const int units = pl->n_slots / smerf::unit_slots(pl->p);
                const int bld = smerf::queue_build(units);
                if (bld < 0) { rc = SMERF_EUNSUPPORTED; break; }
                const int upt = smerf::queue_upt(bld), rmax = smerf::queue_rmax(bld);
                b->h_descs[i].np = (((units + upt - 1) / upt + 31) / 32) * 32;
                const size_t sm = kind == kFF ? smerf_ws_smem_ff(pl, rmax) : smerf_ws_smem_fd(pl, rmax);
                smem = sm > smem ? sm : smem;
                const int n = n_samples[i];
                double total = 0.0;
                for (int sgi = 0; sgi < pl->n_segments; ++sgi)
                    for (int grp = 0; grp < (n + rmax - 1) / rmax; ++grp) {
                        const smerf::Segment& sg = pl->segs_host[sgi];
                        const int r = n - grp * rmax < rmax ? n - grp * rmax : rmax;
                        const double cost = (double)(pl->n_phi / 2) * pl->p * (sg.p1 - sg.p0) * r;
                        total += cost;
                        qs.push_back(std::make_pair(cost, make_int4(i, sgi, grp, (pl->p - 1) * smerf::kQueueBuilds + bld)));
                    }
                // the request's anchor items (smerf::queue_anchor_items of them): both chains, every
                // realisation, blocks of kQueueThreads units
                const int nb = (units + smerf::kQueueThreads - 1) / smerf::kQueueThreads;
                for (int c = 0; c < 2; ++c)
                    for (int r = 0; r < n; ++r)
                        for (int ub = 0; ub < nb; ++ub)
                            qa.push_back(std::make_pair(total, make_int4(i, ub, r, -1 - ((pl->p << 4) | c))));
                // the same in blocks of 128 units, for the anchor launch of the two-launch form
                const int nb128 = (units + 127) / 128;
                for (int c = 0; c < 2; ++c)
                    for (int r = 0; r < n; ++r)
                        for (int ub = 0; ub < nb128; ++ub)
                            qa128.push_back(std::make_pair(total, make_int4(i, ub, r, (pl->p << 4) | c)));
            }
        }
        if (rc != SMERF_OK || (qa.empty() && qs.empty())) continue;
        auto larger = [](const std::pair<double, int4>& x, const std::pair<double, int4>& y) { return x.first > y.first; };
        std::stable_sort(qa.begin(), qa.end(), larger);
        std::stable_sort(qa128.begin(), qa128.end(), larger);
        std::stable_sort(qs.begin(), qs.end(), larger);
        std::vector<int4> anc128;
        for (auto& x : qa128) anc128.push_back(x.second);
        std::vector<int4> items;
        for (auto& x : qa) items.push_back(x.second);
        for (auto& x : qs) items.push_back(x.second);
        Queue q;
        q.kind = kind;
        q.n_anc = (int)qa.size();
        q.n_items = (int)items.size();
        q.n_anc128 = (int)anc128.size();
        q.smem = smem;
        q.ctas = queue_ctas(kind, smem);
        const bool ok = q.ctas > 0 &&
                        smerf::dev_malloc((void**)&q.d_items, sizeof(int4) * q.n_items) == cudaSuccess &&
                        smerf::dev_malloc((void**)&q.d_anc128, sizeof(int4) * (q.n_anc128 ? q.n_anc128 : 1)) == cudaSuccess &&
                        smerf::dev_malloc((void**)&q.d_ctl, sizeof(int) * (2 + n_req)) == cudaSuccess;
        b->queues.push_back(q);
        if (!ok) {
            rc = q.ctas <= 0 ? SMERF_ECUDA : SMERF_ENOMEM;
            break;
        }
        if (cudaMemcpy(q.d_items, items.data(), sizeof(int4) * q.n_items, cudaMemcpyHostToDevice) != cudaSuccess ||
            (q.n_anc128 && cudaMemcpy(q.d_anc128, anc128.data(), sizeof(int4) * q.n_anc128, cudaMemcpyHostToDevice) !=
                               cudaSuccess))
            rc = SMERF_ECUDA;
    }
    if (rc != SMERF_OK) {
        batch_free(b);
        return rc;
    }
    *out = b;
    return SMERF_OK;
}

int smerf_batch_set(smerf_batch* b, const uint64_t* seeds, void* const* outs)
{
    if (!b || (b->n_req > 0 && (!seeds || !outs))) return SMERF_EINVAL;
    for (int i = 0; i < b->n_req; ++i) {
        if (b->counts[i] > 0 && (!outs[i] || ((uintptr_t)outs[i] & 15u))) return SMERF_EINVAL;
        b->seeds[i] = seeds[i];
        b->outs[i] = outs[i];
        b->h_descs[i].seed = seeds[i];
        b->h_descs[i].out = outs[i];
    }
    return SMERF_OK;
}

int smerf_batch_launch(smerf_batch* b, void* stream)
{
    if (!b) return SMERF_EINVAL;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != b->dev) return SMERF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (b->n_req == 0) return SMERF_OK;
    if (!b->singles.empty()) {
        // individually launched requests take their seed and output by value: a captured
        // graph would replay them with the values current at capture, whatever
        // smerf_batch_set changes later, so such batches are not captured
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return SMERF_ECUDA;
        if (cs != cudaStreamCaptureStatusNone) return SMERF_EUNSUPPORTED;
    }
    if (cudaMemcpyAsync(b->d_descs, b->h_descs, sizeof(SampleParams) * b->n_req, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return SMERF_ECUDA;
    const int fail = b->single && b->fail_waits;
    if (b->single) b->fail_waits = 0;
    for (const Queue& q : b->queues) {
        const int rc = launch_queue(q, b->d_descs, b->n_req, b->single, fail, st);
        if (rc != SMERF_OK) return rc;
    }
    for (const Group& g : b->groups) {
        if (queued(g.kind, g.rep->p)) continue;
        const int rc = launch_group(g.kind, g.rep, b->d_descs, g.d_anc, g.n_anc, g.d_seg, g.n_seg, st);
        if (rc != SMERF_OK) return rc;
    }
    for (int i : b->singles) {
        const int rc = smerf_launch_sample(b->plans[i], b->seeds[i], b->counts[i], b->outs[i],
                                           (char*)b->scratch + b->offs[i], st);
        if (rc != SMERF_OK) return rc;
    }
    return SMERF_OK;
}

int smerf_batch_sample(smerf_batch* b, const uint64_t* seeds, void* const* outs, void* stream)
{
    const int rc = smerf_batch_set(b, seeds, outs);
    return rc != SMERF_OK ? rc : smerf_batch_launch(b, stream);
}

int smerf_batch_info(const smerf_batch* b, int* n_groups, int* n_singles)
{
    if (!b) return SMERF_EINVAL;
    if (n_groups) *n_groups = (int)b->groups.size();
    if (n_singles) *n_singles = (int)b->singles.size();
    return SMERF_OK;
}

int smerf_batch_launch_count(const smerf_batch* b)
{
    if (!b) return SMERF_EINVAL;
    int n = 0;
    for (const Queue& q : b->queues)
        n += b->single ? q.n_items > 0 : (q.n_anc128 > 0) + (q.n_items > q.n_anc);
    for (const Group& g : b->groups)
        if (!queued(g.kind, g.rep->p)) n += (g.n_anc > 0) + (g.n_seg > 0);
    for (int i : b->singles) n += smerf_sample_launches(b->plans[i], b->counts[i]);
    return n;
}

int smerf_batch_status(const smerf_batch* b, void* stream)
{
    if (!b) return SMERF_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return SMERF_ECUDA;
    }
    for (const Queue& q : b->queues) {
        int status = 0;
        if (cudaMemcpy(&status, q.d_ctl + 1, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SMERF_ECUDA;
        if (status != 0) return SMERF_ETIMEOUT;
    }
    return SMERF_OK;
}

int smerf_batch_set_single_launch(smerf_batch* b, int single)
{
    if (!b || (single != 0 && single != 1)) return SMERF_EINVAL;
    b->single = single;
    return SMERF_OK;
}

int smerf_debug_batch_fail_waits(smerf_batch* b)
{
    if (!b) return SMERF_EINVAL;
    b->fail_waits = 1;
    return SMERF_OK;
}

int smerf_batch_destroy(smerf_batch* b)
{
    batch_free(b);
    return SMERF_OK;
}

int smerf_sample_batched(const smerf_plan* const* plans, const uint64_t* seeds, const int* n_samples,
                         void* const* outs, int n_req, void* stream)
{
    if (n_req < 0 || (n_req > 0 && (!plans || !seeds || !n_samples || !outs))) return SMERF_EINVAL;
    if (n_req == 0) return SMERF_OK;
    smerf_batch* b = nullptr;
    int rc = smerf_batch_create(plans, n_samples, n_req, &b);
    if (rc != SMERF_OK) return rc;
    rc = smerf_batch_sample(b, seeds, outs, stream);
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess && rc == SMERF_OK) rc = SMERF_ECUDA;
    smerf_batch_destroy(b);
    return rc;
}

}  // extern "C"
