// batch.cu -- the forward path of many detectors as one CUDA graph.
//
// A detector is a plan (its own lmax, kmax, ring grid, precision) with its own
// sky, beam, cube buffer and pointing stream.  The batch captures, once, the
// synth_spin_maps + interp_tod calls of every detector into a CUDA graph whose
// branches are spread over a few streams (longest-processing-time-first
// assignment), so that small detectors overlap and one graph launch replaces
// every per-detector launch.  Optionally it tunes first: each detector's sort
// tile width (8, 16 or 32 columns) by timing its own interpolation, then the
// number of branches (1, 2, 4, 8) by timing replays.
//
// Persistent mode (SL_BATCH_PERSISTENT; SL_FP32 plans, one interpolation
// order): the graph holds persistent contraction launches over every
// detector's blocks (k_lcontract_f32_batch, one launch per number of ring
// pairs per thread among the detectors, side by side: warps take work items
// from a device counter, largest first), each detector's ring FFT and pointing
// sort, and one persistent interpolation launch over every detector's work
// items (k_interp_f32_cells with per-detector arguments).  Its autotuner picks,
// per detector, the contraction's ring pairs per thread and the ring FFT's
// tile by timing the detector's cube build, then one sort-tile width (8, 16,
// 32) for all detectors by timing graph replays.
//
// This layer is host code on top of the plan API; it only adds the plans'
// batch_refs lock, which stops a plan from reallocating scratch that a graph
// still points into.
#include <algorithm>
#include <vector>

#include "sl_internal.cuh"

struct sl_batch {
    int device = 0;
    cudaStream_t stream = nullptr;       // where the graph is captured and replayed
    bool own_stream = false;
    std::vector<sl_batch_item> items;
    std::vector<double> cost;            // per item: measured ms (autotune) or a flop estimate
    std::vector<cudaStream_t> branches;  // capture-only streams
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> joins;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int nstreams = 0;
    double tuned_ms = 0.0, serial_ms = 0.0;
    bool locked = false;
    // persistent mode
    bool persistent = false;
    sl::LcBatchItem *d_items = nullptr;  // contraction work items (device), grouped by ring pairs per thread
    int group_items[sl::kLcBatchGroups] = {};
    unsigned *d_ctr = nullptr;           // work counters: the contraction groups', then the interpolation's
    cudaStream_t lc_side[sl::kLcBatchGroups] = {};   // capture-only streams of the contraction groups
    cudaEvent_t lc_ready = nullptr, lc_done[sl::kLcBatchGroups] = {};
    cudaEvent_t idone[sl::kLcBatchGroups] = {};      // a group's interpolation done
    std::vector<cudaEvent_t> fft_done;               // [group][branch]: a group's FFTs dealt so far
    double group_cost[sl::kLcBatchGroups] = {};       // recurrence steps x ring pairs per group
    int *d_err = nullptr;                // flag of the interpolation's bounded waits
};

namespace sl {

static void destroy_graph(cudaGraph_t &g, cudaGraphExec_t &e) {
    if (e) cudaGraphExecDestroy(e);
    if (g) cudaGraphDestroy(g);
    e = nullptr;
    g = nullptr;
}

// One detector's forward path on its plan's current stream.
static sl_status run_item(const sl_batch_item &it) {
    sl_status st = synth_spin_maps(it.plan, it.sky, it.beam, it.maps);
    if (st != SL_OK) return st;
    return interp_tod(it.plan, it.maps, it.theta, it.phi, it.psi, it.n, it.tod);
}

// Moves every plan to stream s (synchronising the old streams), or back to
// the saved streams when s == nullptr and saved is given.
static sl_status move_plans(sl_batch *b, const std::vector<cudaStream_t> *assign_streams,
                            const std::vector<cudaStream_t> *saved) {
    for (size_t i = 0; i < b->items.size(); ++i) {
        cudaStream_t s = saved ? (*saved)[i] : (*assign_streams)[i];
        sl_status st = sl_plan_set_stream(b->items[i].plan, (void *)s);
        if (st != SL_OK) return st;
    }
    return SL_OK;
}

// Longest processing time first over nbr branches.
static std::vector<int> assign_branches(const sl_batch *b, int nbr) {
    const int n = (int)b->items.size();
    std::vector<int> order(n), br(n, 0);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->cost[x] > b->cost[y]; });
    std::vector<double> load(nbr, 0.0);
    for (int i : order) {
        int best = 0;
        for (int s = 1; s < nbr; ++s)
            if (load[s] < load[best]) best = s;
        br[i] = best;
        load[best] += b->cost[i];
    }
    return br;
}

// Captures the batch with nbr branches into (graph, exec).
static sl_status capture(sl_batch *b, int nbr, cudaGraph_t *graph, cudaGraphExec_t *exec) {
    *graph = nullptr;
    *exec = nullptr;
    const int n = (int)b->items.size();
    const std::vector<int> br = assign_branches(b, nbr);
    std::vector<cudaStream_t> saved(n), target(n);
    std::vector<bool> timing(n);
    for (int i = 0; i < n; ++i) {
        saved[i] = b->items[i].plan->stream;
        target[i] = b->branches[br[i]];
        timing[i] = b->items[i].plan->timing;
    }
    sl_status st = move_plans(b, &target, nullptr);
    if (st != SL_OK) {
        move_plans(b, nullptr, &saved);
        return st;
    }
    for (int i = 0; i < n; ++i) b->items[i].plan->timing = false;   // no event records inside the graph
    st = cuda_check(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (st == SL_OK) {
        sl_status cst = cuda_check(cudaEventRecord(b->fork, b->stream), "fork");
        for (int s = 0; s < nbr && cst == SL_OK; ++s)
            cst = cuda_check(cudaStreamWaitEvent(b->branches[s], b->fork, 0), "fork wait");
        for (int i = 0; i < n && cst == SL_OK; ++i) cst = run_item(b->items[i]);
        for (int s = 0; s < nbr && cst == SL_OK; ++s) {
            cst = cuda_check(cudaEventRecord(b->joins[s], b->branches[s]), "join");
            if (cst == SL_OK) cst = cuda_check(cudaStreamWaitEvent(b->stream, b->joins[s], 0), "join wait");
        }
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (cst == SL_OK) cst = cuda_check(e, "end capture");
        if (cst == SL_OK) cst = cuda_check(cudaGraphInstantiate(exec, g, 0), "graph instantiate");
        if (cst != SL_OK) {
            if (*exec) cudaGraphExecDestroy(*exec);
            if (g) cudaGraphDestroy(g);
            *exec = nullptr;
            g = nullptr;
            cudaGetLastError();
        }
        *graph = g;
        st = cst;
    }
    for (int i = 0; i < n; ++i) b->items[i].plan->timing = timing[i];
    const sl_status rst = move_plans(b, nullptr, &saved);
    return st != SL_OK ? st : rst;
}

// Captures the persistent form (every plan moved to the batch stream meanwhile).
static sl_status capture_persistent(sl_batch *b, cudaGraph_t *graph, cudaGraphExec_t *exec) {
    *graph = nullptr;
    *exec = nullptr;
    const int n = (int)b->items.size();
    std::vector<cudaStream_t> saved(n), here(n, b->stream);
    std::vector<bool> timing(n);
    std::vector<sl_plan *> plans(n);
    std::vector<const double *> sky(n), beam(n);
    int kmax = 0;
    for (int i = 0; i < n; ++i) {
        saved[i] = b->items[i].plan->stream;
        timing[i] = b->items[i].plan->timing;
        plans[i] = b->items[i].plan;
        sky[i] = b->items[i].sky;
        beam[i] = b->items[i].beam;
        kmax = std::max(kmax, plans[i]->K);
    }
    sl_status st = move_plans(b, &here, nullptr);
    if (st != SL_OK) {
        move_plans(b, nullptr, &saved);
        return st;
    }
    for (int i = 0; i < n; ++i) plans[i]->timing = false;   // no event records inside the graph
    st = cuda_check(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (st == SL_OK) {
        // The pointing sorts depend on the pointings only: they run on side branches
        // while the persistent contraction runs on the batch stream; each ring FFT
        // follows the contraction on a branch; the persistent interpolation waits
        // for every branch.
        const int nbr = (int)b->branches.size();
        sl_status cst = cuda_check(cudaEventRecord(b->fork, b->stream), "fork");
        for (int s = 0; s < nbr && cst == SL_OK; ++s)
            cst = cuda_check(cudaStreamWaitEvent(b->branches[s], b->fork, 0), "fork wait");
        std::vector<TiledArgs> args[kLcBatchGroups];   // interpolation arguments per contraction group
        int gkmax[kLcBatchGroups] = {0, 0, 0};
        for (int i = 0; i < n && cst == SL_OK; ++i) {
            const sl_batch_item &it = b->items[i];
            if (it.n == 0) continue;
            plans[i]->stream = b->branches[i % nbr];   // inside the capture: no stream switch that synchronises
            cst = launch_sort_into(plans[i], plans[i]->sort, it.theta, it.phi, it.psi, it.n, 1, 0, 1);
            const int g = lcontract_f32_group(plans[i]);
            args[g].push_back(fine_tiled_args(plans[i], plans[i]->sort, it.maps, it.tod));
            gkmax[g] = std::max(gkmax[g], plans[i]->K);
        }
        if (cst == SL_OK)
            cst = launch_lcontract_f32_batch(b->stream, b->lc_side, b->lc_done, b->lc_ready, plans.data(), sky.data(),
                                             beam.data(), n, b->d_items, b->group_items, b->d_ctr);
        // Per contraction group, in the order the groups are expected to end (least
        // work first): each detector's ring FFT waits for its own group's contraction
        // launch only (the FFTs run on the SMs that the group's CTAs leave while the
        // other groups still run), dealt round-robin over the branches; then one
        // persistent interpolation launch over the group's detectors on the group's
        // stream, after the branches' work so far (their sorts and the group's FFTs).
        int gorder[kLcBatchGroups] = {0, 1, 2};
        std::sort(gorder, gorder + kLcBatchGroups, [&](int x, int y) { return b->group_cost[x] < b->group_cost[y]; });
        int dealt = 0;
        for (int gi = 0; gi < kLcBatchGroups && cst == SL_OK; ++gi) {
            const int g = gorder[gi];
            if (b->group_items[g] == 0) continue;
            for (int i = 0; i < n && cst == SL_OK; ++i) {
                if (lcontract_f32_group(plans[i]) != g) continue;
                const cudaStream_t br = b->branches[dealt++ % nbr];
                cst = cuda_check(cudaStreamWaitEvent(br, b->lc_done[g], 0), "contraction group wait");
                plans[i]->stream = br;
                if (cst == SL_OK) cst = launch_ringfft_synth(plans[i], b->items[i].maps);
            }
            if (args[g].empty()) continue;
            for (int s2 = 0; s2 < nbr && cst == SL_OK; ++s2) {
                cudaEvent_t ev = b->fft_done[g * nbr + s2];
                cst = cuda_check(cudaEventRecord(ev, b->branches[s2]), "ffts of a group");
                if (cst == SL_OK) cst = cuda_check(cudaStreamWaitEvent(b->lc_side[g], ev, 0), "ffts of a group wait");
            }
            if (cst == SL_OK)
                cst = launch_interp_f32_cells(b->lc_side[g], b->device, args[g].data(), (int)args[g].size(),
                                              plans[0]->geom.tile_cols, plans[0]->p, gkmax[g],
                                              b->d_ctr + kLcBatchGroups + g, b->d_err);
            if (cst == SL_OK) cst = cuda_check(cudaEventRecord(b->idone[g], b->lc_side[g]), "interpolation of a group");
        }
        for (int s2 = 0; s2 < nbr && cst == SL_OK; ++s2) {
            cst = cuda_check(cudaEventRecord(b->joins[s2], b->branches[s2]), "join");
            if (cst == SL_OK) cst = cuda_check(cudaStreamWaitEvent(b->stream, b->joins[s2], 0), "join wait");
        }
        for (int g = 0; g < kLcBatchGroups && cst == SL_OK; ++g)   // every group stream joins the batch stream
            if (b->group_items[g] > 0)
                cst = cuda_check(cudaStreamWaitEvent(b->stream, args[g].empty() ? b->lc_done[g] : b->idone[g], 0),
                                 "group join");
        for (int i = 0; i < n; ++i) plans[i]->stream = b->stream;
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (cst == SL_OK) cst = cuda_check(e, "end capture");
        if (cst == SL_OK) cst = cuda_check(cudaGraphInstantiate(exec, g, 0), "graph instantiate");
        if (cst != SL_OK) {
            if (*exec) cudaGraphExecDestroy(*exec);
            if (g) cudaGraphDestroy(g);
            *exec = nullptr;
            g = nullptr;
            cudaGetLastError();
        }
        *graph = g;
        st = cst;
    }
    for (int i = 0; i < n; ++i) plans[i]->timing = timing[i];
    const sl_status rst = move_plans(b, nullptr, &saved);
    return st != SL_OK ? st : rst;
}

// Milliseconds of `reps` replays of exec on the batch stream (after one warm replay).
static sl_status time_replays(sl_batch *b, cudaGraphExec_t exec, int reps, double *ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sl_status st = cuda_check(cudaEventCreate(&e0), "event");
    if (st == SL_OK) st = cuda_check(cudaEventCreate(&e1), "event");
    if (st == SL_OK) st = cuda_check(cudaGraphLaunch(exec, b->stream), "graph launch");
    if (st == SL_OK) st = cuda_check(cudaEventRecord(e0, b->stream), "event");
    for (int r = 0; r < reps && st == SL_OK; ++r) st = cuda_check(cudaGraphLaunch(exec, b->stream), "graph launch");
    if (st == SL_OK) st = cuda_check(cudaEventRecord(e1, b->stream), "event");
    if (st == SL_OK) st = cuda_check(cudaEventSynchronize(e1), "event sync");
    float t = 0.f;
    if (st == SL_OK) st = cuda_check(cudaEventElapsedTime(&t, e0, e1), "elapsed");
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    *ms = (double)t / reps;
    return st;
}

// Milliseconds of fn() enqueued on the batch stream (plans moved there by the caller).
template <typename F>
static sl_status time_on_stream(sl_batch *b, F fn, double *ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sl_status st = cuda_check(cudaEventCreate(&e0), "event");
    if (st == SL_OK) st = cuda_check(cudaEventCreate(&e1), "event");
    if (st == SL_OK) st = cuda_check(cudaEventRecord(e0, b->stream), "event");
    if (st == SL_OK) st = fn();
    if (st == SL_OK) st = cuda_check(cudaEventRecord(e1, b->stream), "event");
    if (st == SL_OK) st = cuda_check(cudaEventSynchronize(e1), "event sync");
    float t = 0.f;
    if (st == SL_OK) st = cuda_check(cudaEventElapsedTime(&t, e0, e1), "elapsed");
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    *ms = (double)t;
    return st;
}

// Per detector: the fastest tile width for its own pointings, and its cost;
// then the serial time of the whole batch.
static sl_status autotune_items(sl_batch *b) {
    const int n = (int)b->items.size();
    for (int i = 0; i < n; ++i) {
        const sl_batch_item &it = b->items[i];
        double t_syn = 0.0;
        sl_status st = time_on_stream(b, [&] { return synth_spin_maps(it.plan, it.sky, it.beam, it.maps); }, &t_syn);
        if (st != SL_OK) return st;
        int best_tc = it.plan->geom.tile_cols;
        double best = -1.0;
        for (int tc : {8, 16, 32}) {
            if (sl_plan_set_tile_cols(it.plan, tc) != SL_OK) continue;   // not valid for this grid
            auto interp = [&] { return interp_tod(it.plan, it.maps, it.theta, it.phi, it.psi, it.n, it.tod); };
            double t = 0.0;
            if ((st = time_on_stream(b, interp, &t)) != SL_OK) return st;   // warm
            if ((st = time_on_stream(b, interp, &t)) != SL_OK) return st;
            if (best < 0.0 || t < best) {
                best = t;
                best_tc = tc;
            }
        }
        if ((st = sl_plan_set_tile_cols(it.plan, best_tc)) != SL_OK) return st;
        b->cost[i] = t_syn + std::max(best, 0.0);
    }
    return time_on_stream(b, [&] {
        for (const sl_batch_item &it : b->items) {
            sl_status s = run_item(it);
            if (s != SL_OK) return s;
        }
        return SL_OK;
    }, &b->serial_ms);
}

// Persistent mode, per detector: the contraction's ring pairs per thread and
// the ring FFT tile by timing its cube build (plans moved to the batch stream
// by the caller).
static sl_status autotune_synth(sl_batch *b) {
    for (const sl_batch_item &it : b->items) {
        sl_plan *p = it.plan;
        auto synth = [&] { return synth_spin_maps(p, it.sky, it.beam, it.maps); };
        double t = 0.0, best = -1.0;
        sl_status st;
        int best_ppt = 0;
        for (int ppt : {8, 4, 2}) {
            if (sl_plan_set_contraction_pairs(p, ppt) != SL_OK) continue;
            if ((st = time_on_stream(b, synth, &t)) != SL_OK) return st;   // warm
            if ((st = time_on_stream(b, synth, &t)) != SL_OK) return st;
            if (best < 0.0 || t < best) {
                best = t;
                best_ppt = ppt;
            }
        }
        if ((st = sl_plan_set_contraction_pairs(p, best_ppt)) != SL_OK) return st;
        best = -1.0;
        int brg = 0, bkg = 0;
        for (int rg : {1, 2, 4})
            for (int kg : {1, 2}) {
                if (sl_plan_set_fft_tile(p, rg, kg) != SL_OK) continue;   // not valid for this grid
                if ((st = time_on_stream(b, synth, &t)) != SL_OK) return st;
                if (best < 0.0 || t < best) {
                    best = t;
                    brg = rg;
                    bkg = kg;
                }
            }
        if ((st = sl_plan_set_fft_tile(p, brg, bkg)) != SL_OK) return st;
    }
    return SL_OK;
}

static void release(sl_batch *b) {
    if (b->locked)
        for (const sl_batch_item &it : b->items) --it.plan->batch_refs;
    b->locked = false;
    destroy_graph(b->graph, b->exec);
    for (cudaStream_t s : b->branches) cudaStreamDestroy(s);
    b->branches.clear();
    for (cudaStream_t s : b->lc_side)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->lc_done)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : b->idone)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : b->fft_done)
        if (e) cudaEventDestroy(e);
    b->fft_done.clear();
    if (b->lc_ready) cudaEventDestroy(b->lc_ready);
    if (b->fork) cudaEventDestroy(b->fork);
    for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
    b->joins.clear();
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_ctr) cudaFree(b->d_ctr);
    if (b->d_err) cudaFree(b->d_err);
    b->d_items = nullptr;
    b->d_ctr = nullptr;
    b->d_err = nullptr;
}

// Persistent mode: validation, a common tile width, the batch's device
// counters and the contraction groups' streams.
static sl_status prepare_persistent(sl_batch *b) {
    const int n = (int)b->items.size();
    if (n > kMaxBatchDets)
        return set_error(SL_ERR_UNSUPPORTED, "persistent batch: %d detectors, at most %d", n, kMaxBatchDets);
    int tc = 32;
    for (int i = 0; i < n; ++i) {
        const sl_plan *p = b->items[i].plan;
        if (p->precision != SL_FP32)
            return set_error(SL_ERR_UNSUPPORTED, "persistent batch: item %d is not an SL_FP32 plan", i);
        if (p->p != b->items[0].plan->p)
            return set_error(SL_ERR_UNSUPPORTED, "persistent batch: items 0 and %d differ in interp_order", i);
        tc = std::min(tc, p->geom.tile_cols);
    }
    for (int i = 0; i < n; ++i) {   // one tile width for the shared interpolation launch
        sl_status st = sl_plan_set_tile_cols(b->items[i].plan, tc);
        if (st != SL_OK) return st;
    }
    sl_status st = cuda_check(cudaMalloc(&b->d_ctr, 2 * kLcBatchGroups * sizeof(unsigned)), "batch counters");
    for (int j = 0; j < kLcBatchGroups && st == SL_OK; ++j) {
        st = cuda_check(cudaStreamCreateWithFlags(&b->lc_side[j], cudaStreamNonBlocking), "contraction stream");
        if (st == SL_OK) st = cuda_check(cudaEventCreateWithFlags(&b->lc_done[j], cudaEventDisableTiming), "event");
        if (st == SL_OK) st = cuda_check(cudaEventCreateWithFlags(&b->idone[j], cudaEventDisableTiming), "event");
    }
    b->fft_done.assign(kLcBatchGroups * b->branches.size(), nullptr);
    for (size_t j = 0; j < b->fft_done.size() && st == SL_OK; ++j)
        st = cuda_check(cudaEventCreateWithFlags(&b->fft_done[j], cudaEventDisableTiming), "event");
    if (st == SL_OK) st = cuda_check(cudaEventCreateWithFlags(&b->lc_ready, cudaEventDisableTiming), "event");
    if (st == SL_OK) st = cuda_check(cudaMalloc(&b->d_err, sizeof(int)), "batch error flag");
    if (st == SL_OK) st = cuda_check(cudaMemset(b->d_err, 0, sizeof(int)), "batch error flag");
    return st;
}

// (Re)builds the contraction's work items from the plans' current settings.
static sl_status upload_items(sl_batch *b) {
    std::vector<sl_plan *> plans;
    for (const sl_batch_item &it : b->items) plans.push_back(it.plan);
    std::vector<LcBatchItem> items;
    sl_status st = lcontract_f32_batch_items(plans.data(), (int)plans.size(), items, b->group_items);
    if (st != SL_OK) return st;
    for (int g = 0; g < kLcBatchGroups; ++g) b->group_cost[g] = 0.0;
    for (const LcBatchItem &it : items) b->group_cost[it.ppt == 8 ? 0 : (it.ppt == 4 ? 1 : 2)] += it.cost;
    if (b->d_items) cudaFree(b->d_items);
    b->d_items = nullptr;
    st = cuda_check(cudaMalloc(&b->d_items, items.size() * sizeof(LcBatchItem)), "batch work items");
    if (st == SL_OK)
        st = cuda_check(cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(LcBatchItem), cudaMemcpyHostToDevice),
                        "batch work items");
    return st;
}

}  // namespace sl

using namespace sl;

extern "C" {

sl_status sl_batch_create(sl_batch **out, const sl_batch_item *items, int nitems, void *stream, int flags) {
    if (!out) return set_error(SL_ERR_ARG, "sl_batch_create: out is NULL");
    *out = nullptr;
    if (!items || nitems < 1) return set_error(SL_ERR_ARG, "sl_batch_create: no items");
    for (int i = 0; i < nitems; ++i) {
        const sl_batch_item &it = items[i];
        if (!it.plan) return set_error(SL_ERR_ARG, "sl_batch_create: item %d has no plan", i);
        if (it.plan->device != items[0].plan->device)
            return set_error(SL_ERR_ARG, "sl_batch_create: item %d is on device %d, item 0 on %d", i,
                             it.plan->device, items[0].plan->device);
        for (int j = 0; j < i; ++j)
            if (items[j].plan == it.plan)
                return set_error(SL_ERR_ARG, "sl_batch_create: items %d and %d share a plan", j, i);
        if (!it.sky || !it.beam || !it.maps) return set_error(SL_ERR_ARG, "sl_batch_create: item %d: NULL buffer", i);
        if (it.n < 0 || it.n >= ((int64_t)1 << 31))
            return set_error(SL_ERR_ARG, "sl_batch_create: item %d: n=%lld outside [0, 2^31)", i, (long long)it.n);
        if (it.n > 0 && (!it.theta || !it.phi || !it.psi || !it.tod))
            return set_error(SL_ERR_ARG, "sl_batch_create: item %d: NULL pointing or TOD buffer", i);
    }
    sl_batch *b = new (std::nothrow) sl_batch();
    if (!b) return set_error(SL_ERR_NOMEM, "sl_batch_create: host allocation");
    b->device = items[0].plan->device;
    b->items.assign(items, items + nitems);
    b->cost.assign(nitems, 0.0);
    sl_status st = cuda_check(cudaSetDevice(b->device), "cudaSetDevice");
    if (st == SL_OK && stream) {
        b->stream = (cudaStream_t)stream;
    } else if (st == SL_OK) {   // the legacy stream cannot be captured: a blocking stream of our own
        st = cuda_check(cudaStreamCreate(&b->stream), "batch stream");
        b->own_stream = st == SL_OK;
    }
    const int max_branches = std::min(8, nitems);
    for (int s = 0; s < max_branches && st == SL_OK; ++s) {
        cudaStream_t bs = nullptr;
        st = cuda_check(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking), "branch stream");
        if (st == SL_OK) b->branches.push_back(bs);
        cudaEvent_t ev = nullptr;
        if (st == SL_OK) st = cuda_check(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "join event");
        if (st == SL_OK) b->joins.push_back(ev);
    }
    if (st == SL_OK) st = cuda_check(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "fork event");
    for (int i = 0; i < nitems && st == SL_OK; ++i) st = sl_plan_reserve(b->items[i].plan, b->items[i].n);
    for (int i = 0; i < nitems && st == SL_OK; ++i) {   // flop estimate (FP64 at 1/64 of the FP32 rate)
        const sl_plan *p = b->items[i].plan;
        const double w = p->precision == SL_FP64 ? 64.0 : (p->precision == SL_DF64 ? 12.0 : 1.0);
        b->cost[i] = w * (11.0 * (double)p->lsteps + 4.0 * 16.0 * (p->K + 1) * (double)b->items[i].n);
    }
    if (st == SL_OK && (flags & SL_BATCH_PERSISTENT)) {
        b->persistent = true;
        st = prepare_persistent(b);
        if (st == SL_OK && (flags & SL_BATCH_AUTOTUNE)) {
            std::vector<cudaStream_t> saved(nitems), here(nitems, b->stream);
            for (int i = 0; i < nitems; ++i) saved[i] = b->items[i].plan->stream;
            st = move_plans(b, &here, nullptr);
            if (st == SL_OK) st = autotune_synth(b);
            if (st == SL_OK)   // the detectors one after another (their own kernels), for reference
                st = time_on_stream(b, [&] {
                    for (const sl_batch_item &it : b->items) {
                        sl_status s2 = run_item(it);
                        if (s2 != SL_OK) return s2;
                    }
                    return SL_OK;
                }, &b->serial_ms);
            const sl_status rst = move_plans(b, nullptr, &saved);
            if (st == SL_OK) st = rst;
            // one tile width for all detectors, by timing graph replays
            int best_tc = 0;
            if (st == SL_OK) st = upload_items(b);
            for (int tc : {32, 16, 8}) {
                if (st != SL_OK) break;
                bool ok = true;
                for (const sl_batch_item &it : b->items) ok = ok && sl_plan_set_tile_cols(it.plan, tc) == SL_OK;
                if (!ok) continue;
                cudaGraph_t g = nullptr;
                cudaGraphExec_t e = nullptr;
                double ms = 0.0;
                st = capture_persistent(b, &g, &e);
                if (st == SL_OK) st = time_replays(b, e, 2, &ms);
                if (st == SL_OK && (best_tc == 0 || ms < b->tuned_ms)) {
                    best_tc = tc;
                    b->tuned_ms = ms;
                }
                destroy_graph(g, e);
            }
            if (st == SL_OK && best_tc == 0) st = set_error(SL_ERR_UNSUPPORTED, "persistent batch: no common tile width");
            for (const sl_batch_item &it : b->items)   // settle on it (re-tiles) and capture once more
                if (st == SL_OK) st = sl_plan_set_tile_cols(it.plan, best_tc);
            b->nstreams = 1;
            if (st == SL_OK) st = capture_persistent(b, &b->graph, &b->exec);
        } else if (st == SL_OK) {
            b->nstreams = 1;
            st = upload_items(b);
            if (st == SL_OK) st = capture_persistent(b, &b->graph, &b->exec);
        }
    } else if (st == SL_OK && (flags & SL_BATCH_AUTOTUNE)) {
        std::vector<cudaStream_t> saved(nitems), here(nitems, b->stream);
        for (int i = 0; i < nitems; ++i) saved[i] = b->items[i].plan->stream;
        st = move_plans(b, &here, nullptr);
        if (st == SL_OK) st = autotune_items(b);
        const sl_status rst = move_plans(b, nullptr, &saved);
        if (st == SL_OK) st = rst;
        for (int nbr = 1; nbr <= max_branches && st == SL_OK; nbr *= 2) {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t e = nullptr;
            double ms = 0.0;
            st = capture(b, nbr, &g, &e);
            if (st == SL_OK) st = time_replays(b, e, 2, &ms);
            if (st == SL_OK && (b->nstreams == 0 || ms < b->tuned_ms)) {
                destroy_graph(b->graph, b->exec);
                b->graph = g;
                b->exec = e;
                b->nstreams = nbr;
                b->tuned_ms = ms;
            } else {
                destroy_graph(g, e);
            }
        }
    } else if (st == SL_OK) {
        b->nstreams = std::min(4, max_branches);
        st = capture(b, b->nstreams, &b->graph, &b->exec);
    }
    if (st == SL_OK) {
        for (const sl_batch_item &it : b->items) ++it.plan->batch_refs;
        b->locked = true;
        *out = b;
        return SL_OK;
    }
    release(b);
    delete b;
    return st;
}

sl_status sl_batch_run(sl_batch *b) {
    if (!b || !b->exec) return set_error(SL_ERR_ARG, "sl_batch_run: no batch");
    sl_status st = cuda_check(cudaSetDevice(b->device), "cudaSetDevice");
    if (st != SL_OK) return st;
    return cuda_check(cudaGraphLaunch(b->exec, b->stream), "sl_batch_run: graph launch");
}

sl_status sl_batch_sync(sl_batch *b) {
    if (!b) return set_error(SL_ERR_ARG, "sl_batch_sync: no batch");
    sl_status st = cuda_check(cudaSetDevice(b->device), "cudaSetDevice");
    if (st == SL_OK) st = cuda_check(cudaStreamSynchronize(b->stream), "sl_batch_sync");
    if (st != SL_OK || !b->d_err) return st;
    int flag = 0;
    if ((st = cuda_check(cudaMemcpy(&flag, b->d_err, sizeof(int), cudaMemcpyDeviceToHost), "batch error flag")) != SL_OK)
        return st;
    if (flag) {
        cudaMemset(b->d_err, 0, sizeof(int));
        return set_error(SL_ERR_TIMEOUT, "a bounded wait of the batch's interpolation expired");
    }
    return SL_OK;
}

sl_status sl_batch_get_info(const sl_batch *b, sl_batch_info *info) {
    if (!b || !info) return set_error(SL_ERR_ARG, "sl_batch_get_info: NULL argument");
    info->nitems = (int)b->items.size();
    info->nstreams = b->nstreams;
    info->persistent = b->persistent ? 1 : 0;
    info->tuned_ms = b->tuned_ms;
    info->serial_ms = b->serial_ms;
    info->kernel_nodes = info->graph_nodes = 0;
    size_t count = 0;
    sl_status st = cuda_check(cudaGraphGetNodes(b->graph, nullptr, &count), "graph nodes");
    if (st != SL_OK) return st;
    std::vector<cudaGraphNode_t> nodes(count);
    if (count && (st = cuda_check(cudaGraphGetNodes(b->graph, nodes.data(), &count), "graph nodes")) != SL_OK)
        return st;
    info->graph_nodes = (int)count;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++info->kernel_nodes;
    }
    return SL_OK;
}

void sl_batch_destroy(sl_batch *b) {
    if (!b) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    release(b);
    delete b;
    cudaSetDevice(prev);
}

}  // extern "C"
