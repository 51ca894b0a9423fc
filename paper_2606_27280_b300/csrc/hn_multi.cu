// Batched serving (an extension of the method): many query batches of uneven
// sizes against several indexes in one call, and the autotuner that picks the
// scan kind and dense work-unit size per index.
//
// hn_search_multi groups the batches by index and concatenates each group's
// queries, so that small batches share the dense scan's 256-query units.  The
// groups whose indexes share the dense tile format run their one-pass scans as
// ONE persistent launch over all of them (work units numbered group by group),
// with query preparation before it and each group's threshold, survivor
// extraction and rescore after it on the group's own stream; any other group
// runs the whole search pipeline on its stream.  The set is captured once into
// a CUDA graph (fork / join across the streams) and the instantiated graph is
// replayed while the same set of batches comes back.  Per-batch completion
// times come from events recorded inside the graph.
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "hn_internal.cuh"

namespace hn {

struct Group {
    hn_index *h = nullptr;
    Index *ix = nullptr;
    std::vector<int32_t> bids;   // batches of this group, in call order
    std::vector<int64_t> off;    // their first row in the concatenated arrays
    int64_t Q = 0;
    int scan = HN_SCAN_STREAM;
    int32_t cap = 0;
    float *qcat = nullptr;
    int64_t *icat = nullptr;
    double *scat = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;   // join dependency
    cudaEvent_t stamp = nullptr;  // completion time (a real event record, also inside a graph)
    int joined = -1;              // position in the shared one-pass scan, or -1
    cudaEvent_t prepped = nullptr;  // joined: query preparation done
};

struct Plan {
    std::vector<uint64_t> key;           // what the graph was built for
    std::vector<Group> groups;
    std::vector<int32_t> batch_group;
    std::vector<uint64_t> gens;          // workspace generation of each group's index at capture
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t start = nullptr, fork = nullptr, scanned = nullptr;
    DenseMulti *dm = nullptr;            // the shared one-pass scan of the joined groups
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool valid = false;
};

static std::mutex g_mu;
static Plan g_plan;

static void release_plan(Plan &p) {
    for (Group &g : p.groups) {
        cudaFree(g.qcat);
        cudaFree(g.icat);
        cudaFree(g.scat);
        if (g.st) cudaStreamDestroy(g.st);
        if (g.done) cudaEventDestroy(g.done);
        if (g.stamp) cudaEventDestroy(g.stamp);
        if (g.prepped) cudaEventDestroy(g.prepped);
    }
    p.groups.clear();
    dense_multi_destroy(p.dm);
    p.dm = nullptr;
    if (p.exec) cudaGraphExecDestroy(p.exec);
    if (p.graph) cudaGraphDestroy(p.graph);
    p.exec = nullptr;
    p.graph = nullptr;
    p.valid = false;
}

static std::vector<uint64_t> make_key(const hn_batch *b, int32_t nb) {
    std::vector<uint64_t> k;
    k.reserve((size_t)nb * 6);
    for (int32_t i = 0; i < nb; ++i) {
        k.push_back((uint64_t)(uintptr_t)b[i].index);
        k.push_back(index_state(b[i].index)->serial);
        k.push_back((uint64_t)(uintptr_t)b[i].q);
        k.push_back((uint64_t)b[i].nq);
        k.push_back((uint64_t)(uintptr_t)b[i].out_idx);
        k.push_back((uint64_t)(uintptr_t)b[i].out_sim);
    }
    return k;
}

// Enqueue the whole set: fork from `s0`, one stream per group, join back on `s0`.
static hn_status enqueue_plan(Plan &p, const hn_batch *b, cudaStream_t s0, bool capturing) {
    // while capturing, timing records are external so that the graph keeps them as
    // event-record nodes (outside a capture the flag is not accepted)
    const unsigned rec = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    HN_CUDA(cudaEventRecordWithFlags(p.start, s0, rec));
    HN_CUDA(cudaEventRecord(p.fork, s0));
    auto finish = [&](Group &g) -> hn_status {
        for (size_t j = 0; j < g.bids.size(); ++j) {
            const hn_batch &x = b[g.bids[j]];
            if (!x.nq) continue;
            HN_CUDA(cudaMemcpyAsync(x.out_idx, g.icat + g.off[j], sizeof(int64_t) * x.nq, cudaMemcpyDeviceToDevice,
                                    g.st));
            HN_CUDA(cudaMemcpyAsync(x.out_sim, g.scat + g.off[j], sizeof(double) * x.nq, cudaMemcpyDeviceToDevice,
                                    g.st));
        }
        HN_CUDA(cudaEventRecordWithFlags(g.stamp, g.st, rec));
        HN_CUDA(cudaEventRecord(g.done, g.st));
        return HN_OK;
    };
    for (Group &g : p.groups) {
        HN_CUDA(cudaStreamWaitEvent(g.st, p.fork, 0));
        for (size_t j = 0; j < g.bids.size(); ++j) {
            const hn_batch &x = b[g.bids[j]];
            if (x.nq)
                HN_CUDA(cudaMemcpyAsync(g.qcat + g.off[j] * kD, x.q, sizeof(float) * kD * x.nq,
                                        cudaMemcpyDeviceToDevice, g.st));
        }
        if (g.joined >= 0) {
            // the first steps of the search pipeline; the scan is shared (below)
            Workspace &ws = g.ix->ws;
            HN_CUDA(cudaMemsetAsync(ws.status, 0, 8 * sizeof(int32_t), g.st));
            HN_CUDA(cudaMemsetAsync(ws.counters, 0, 8 * sizeof(long long), g.st));
            HN_CUDA(launch_query_prep(*g.ix, g.qcat, g.Q, 1.f, g.st));
            HN_CUDA(cudaEventRecord(g.prepped, g.st));
            continue;
        }
        hn_status st = enqueue_search(*g.ix, g.qcat, g.Q, g.scan, nullptr, 4, g.icat, g.scat, false, g.st);
        if (st != HN_OK) return st;
        st = finish(g);
        if (st != HN_OK) return st;
    }
    if (p.dm) {
        // one persistent one-pass scan over every joined group, then each group's own steps
        for (Group &g : p.groups)
            if (g.joined >= 0) HN_CUDA(cudaStreamWaitEvent(s0, g.prepped, 0));
        HN_CUDA(dense_multi_scan(p.dm, s0));
        HN_CUDA(cudaEventRecord(p.scanned, s0));
        for (Group &g : p.groups) {
            if (g.joined < 0) continue;
            Workspace &ws = g.ix->ws;
            HN_CUDA(cudaStreamWaitEvent(g.st, p.scanned, 0));
            HN_CUDA(dense_multi_post(p.dm, g.joined, g.qcat, g.st));
            HN_CUDA(launch_rescore(*g.ix, g.qcat, g.Q, g.icat, g.scat, g.st));
            HN_CUDA(cudaMemcpyAsync(ws.h_status, ws.status, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, g.st));
            HN_CUDA(cudaMemcpyAsync(ws.h_status + 8, ws.counters, 8 * sizeof(long long), cudaMemcpyDeviceToHost,
                                    g.st));
            hn_status st = finish(g);
            if (st != HN_OK) return st;
        }
    }
    for (Group &g : p.groups) HN_CUDA(cudaStreamWaitEvent(s0, g.done, 0));
    return HN_OK;
}

// Group the batches, size every index's scratch, allocate the concatenation buffers.
static hn_status build_plan(Plan &p, const hn_batch *b, int32_t nb, const std::map<Index *, int32_t> &caps) {
    release_plan(p);
    HN_CUDA(dense_init());
    std::map<hn_index *, int32_t> gid;
    p.batch_group.assign(nb, -1);
    for (int32_t i = 0; i < nb; ++i) {
        auto it = gid.find(b[i].index);
        if (it == gid.end()) {
            it = gid.emplace(b[i].index, (int32_t)p.groups.size()).first;
            p.groups.emplace_back();
            p.groups.back().h = b[i].index;
            p.groups.back().ix = index_state_mut(b[i].index);
        }
        Group &g = p.groups[it->second];
        g.bids.push_back(i);
        g.off.push_back(g.Q);
        g.Q += b[i].nq;
        p.batch_group[i] = it->second;
    }
    for (Group &g : p.groups) {
        if (g.Q == 0) continue;
        g.scan = pick_scan(*g.ix, g.Q, HN_SCAN_AUTO);
        auto c = caps.find(g.ix);
        g.cap = c != caps.end() ? c->second : default_cap(*g.ix);
        hn_status st = prepare_search(*g.ix, g.Q, g.scan, g.cap);
        if (st != HN_OK) return st;
        HN_CUDA(cudaMalloc(&g.qcat, sizeof(float) * kD * g.Q));
        HN_CUDA(cudaMalloc(&g.icat, sizeof(int64_t) * g.Q));
        HN_CUDA(cudaMalloc(&g.scat, sizeof(double) * g.Q));
        HN_CUDA(cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking));
        HN_CUDA(cudaEventCreate(&g.done));
        HN_CUDA(cudaEventCreate(&g.stamp));
    }
    // drop empty groups (all their batches have nq == 0)
    p.groups.erase(std::remove_if(p.groups.begin(), p.groups.end(), [](const Group &g) { return g.Q == 0; }),
                   p.groups.end());
    for (int32_t i = 0; i < nb; ++i) p.batch_group[i] = -1;
    for (size_t gi = 0; gi < p.groups.size(); ++gi)
        for (int32_t bi : p.groups[gi].bids) p.batch_group[bi] = (int32_t)gi;
    // the dense one-pass groups that share the first such group's tile format run one shared scan
    std::vector<const Index *> jix;
    std::vector<int64_t> jnq;
    int kp = 0;
    bool f8 = false;
    for (Group &g : p.groups) {
        if (g.scan != HN_SCAN_DENSE) continue;
        if (kp == 0) {
            kp = g.ix->k_pad16;
            f8 = g.ix->prefix == HN_PREFIX_FP8_E4M3;
        }
        if (dense_multi_joinable(*g.ix, g.Q, kp, f8)) {
            g.joined = (int)jix.size();
            jix.push_back(g.ix);
            jnq.push_back(g.Q);
        }
    }
    if (jix.size() >= 2) {
        hn_status st = dense_multi_create(jix, jnq, &p.dm);
        if (st != HN_OK) return st;
        for (Group &g : p.groups)
            if (g.joined >= 0) HN_CUDA(cudaEventCreateWithFlags(&g.prepped, cudaEventDisableTiming));
        if (!p.scanned) HN_CUDA(cudaEventCreateWithFlags(&p.scanned, cudaEventDisableTiming));
    } else {
        for (Group &g : p.groups) g.joined = -1;
    }
    p.gens.clear();
    for (Group &g : p.groups) p.gens.push_back(g.ix->ws.gen);
    if (!p.cap_stream) HN_CUDA(cudaStreamCreateWithFlags(&p.cap_stream, cudaStreamNonBlocking));
    if (!p.start) HN_CUDA(cudaEventCreate(&p.start));
    if (!p.fork) HN_CUDA(cudaEventCreate(&p.fork));
    return HN_OK;
}

static bool plan_current(const Plan &p, const std::vector<uint64_t> &key) {
    if (!p.valid || p.key != key) return false;
    for (size_t i = 0; i < p.groups.size(); ++i)
        if (p.groups[i].ix->ws.gen != p.gens[i]) return false;  // scratch reallocated since capture
    return true;
}

}  // namespace hn

using namespace hn;

extern "C" {

hn_status hn_search_multi(const hn_batch *batches, int32_t nb, const hn_multi_opts *opts, hn_multi_stats *stats,
                          void *stream) {
    if (nb < 0 || (nb > 0 && !batches)) return fail(HN_ERR_INVALID_ARG, "bad batch array");
    hn_multi_opts o{};
    o.use_graph = 1;
    if (opts) o = *opts;
    for (int i = 0; i < 7; ++i)
        if (o.reserved[i]) return fail(HN_ERR_INVALID_ARG, "reserved option fields must be zero");
    int64_t total = 0;
    for (int32_t i = 0; i < nb; ++i) {
        const hn_batch &x = batches[i];
        if (!x.index) return fail(HN_ERR_INVALID_ARG, "batch " + std::to_string(i) + ": index is NULL");
        if (x.nq < 0 || x.nq > ((int64_t)1 << 30)) return fail(HN_ERR_INVALID_ARG, "batch " + std::to_string(i) + ": bad nq");
        if (x.nq && (!x.q || !x.out_idx || !x.out_sim || ((uintptr_t)x.q & 15u)))
            return fail(HN_ERR_INVALID_ARG, "batch " + std::to_string(i) + ": null or unaligned pointer");
        total += x.nq;
    }
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->n_queries = total;
        stats->n_batches = nb;
    }
    if (total == 0) return HN_OK;
    std::lock_guard<std::mutex> lock(g_mu);
    Plan &p = g_plan;
    cudaStream_t s = (cudaStream_t)stream;
    const std::vector<uint64_t> key = make_key(batches, nb);
    std::map<Index *, int32_t> caps;
    int32_t reruns = 0;
    bool replayed = false;
    for (;;) {
        if (!plan_current(p, key) || !o.use_graph) {
            hn_status st = build_plan(p, batches, nb, caps);
            if (st != HN_OK) {
                release_plan(p);
                return st;
            }
            p.key = key;
            if (o.use_graph) {
                // capture on a private stream, then replay on the caller's
                HN_CUDA(cudaStreamBeginCapture(p.cap_stream, cudaStreamCaptureModeThreadLocal));
                st = enqueue_plan(p, batches, p.cap_stream, true);
                cudaGraph_t graph = nullptr;
                cudaError_t e = cudaStreamEndCapture(p.cap_stream, &graph);
                if (st != HN_OK) {
                    if (graph) cudaGraphDestroy(graph);
                    release_plan(p);
                    return st;
                }
                if (e != cudaSuccess) {
                    release_plan(p);
                    return cuda_fail(e, "cudaStreamEndCapture");
                }
                p.graph = graph;
                e = cudaGraphInstantiate(&p.exec, p.graph, 0);
                if (e != cudaSuccess) {
                    release_plan(p);
                    return cuda_fail(e, "cudaGraphInstantiate");
                }
            }
            p.valid = true;
        } else {
            replayed = true;
        }
        if (o.use_graph) {
            HN_CUDA(cudaGraphLaunch(p.exec, s));
        } else {
            hn_status st = enqueue_plan(p, batches, s, false);
            if (st != HN_OK) return st;
        }
        HN_CUDA(cudaStreamSynchronize(s));
        bool overflow = false;
        for (Group &g : p.groups) {
            int32_t want = 0;
            hn_status st = check_search(*g.ix, g.Q, &want);
            if (st == HN_ERR_OVERFLOW) {
                overflow = true;
                caps[g.ix] = want;
            } else if (st != HN_OK) {
                return st;
            }
        }
        if (!overflow) break;
        if (reruns >= 2) return fail(HN_ERR_OVERFLOW, "survivor storage overflow after re-runs");
        ++reruns;
        p.valid = false;  // recapture with more survivor slots
    }
    if (stats) {
        stats->n_groups = (int32_t)p.groups.size();
        stats->joined = p.dm ? (int32_t)std::count_if(p.groups.begin(), p.groups.end(),
                                                      [](const Group &g) { return g.joined >= 0; })
                             : 0;
        stats->graph_replayed = replayed ? 1 : 0;
        stats->reruns = reruns;
        std::vector<float> gms(p.groups.size(), 0.f);
        for (size_t gi = 0; gi < p.groups.size(); ++gi) {
            HN_CUDA(cudaEventElapsedTime(&gms[gi], p.start, p.groups[gi].stamp));
            const long long *hc = reinterpret_cast<const long long *>(p.groups[gi].ix->ws.h_status + 8);
            stats->survivors += hc[CT_SURVIVORS];
            stats->ms_total = std::max(stats->ms_total, gms[gi]);
        }
        std::vector<float> lat;
        for (int32_t i = 0; i < nb; ++i)
            if (p.batch_group[i] >= 0) lat.push_back(gms[p.batch_group[i]]);
        std::sort(lat.begin(), lat.end());
        if (!lat.empty()) {
            auto pct = [&](double f) { return lat[std::min(lat.size() - 1, (size_t)(f * (lat.size() - 1) + 0.5))]; };
            stats->batch_ms_p50 = pct(0.50);
            stats->batch_ms_p99 = pct(0.99);
            stats->batch_ms_max = lat.back();
        }
    }
    return HN_OK;
}

hn_status hn_autotune(hn_index *index, const int64_t *sizes, int32_t n_sizes, hn_tune_result *out, void *stream) {
    if (!index || !sizes || n_sizes < 1 || n_sizes > HN_TUNE_MAX) return fail(HN_ERR_INVALID_ARG, "bad arguments");
    Index &ix = *index_state_mut(index);
    for (int32_t i = 0; i < n_sizes; ++i)
        if (sizes[i] < 1 || sizes[i] > ix.n || sizes[i] > (1 << 24)) return fail(HN_ERR_INVALID_ARG, "bad size");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t qmax = 0;
    for (int32_t i = 0; i < n_sizes; ++i) qmax = std::max(qmax, sizes[i]);
    int64_t *oi = nullptr;
    double *os = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    HN_CUDA(cudaMalloc(&oi, sizeof(int64_t) * qmax));
    HN_CUDA(cudaMalloc(&os, sizeof(double) * qmax));
    HN_CUDA(cudaEventCreate(&a));
    HN_CUDA(cudaEventCreate(&b));
    // queries: the index's own first rows (HN-normalised, resident on the device)
    auto time_search = [&](int64_t nq, int scan, float *ms) -> hn_status {
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            int32_t cap = default_cap(ix);
            hn_status st = prepare_search(ix, nq, scan, cap);
            if (st != HN_OK) return st;
            HN_CUDA(cudaEventRecord(a, s));
            st = enqueue_search(ix, ix.rows, nq, scan, nullptr, 4, oi, os, false, s);
            if (st != HN_OK) return st;
            HN_CUDA(cudaEventRecord(b, s));
            HN_CUDA(cudaStreamSynchronize(s));
            int32_t want = 0;
            st = check_search(ix, nq, &want);
            if (st == HN_ERR_OVERFLOW) {
                ix.ws.last_max = want;
                --rep;
                continue;
            }
            if (st != HN_OK) return st;
            float t = 0;
            HN_CUDA(cudaEventElapsedTime(&t, a, b));
            if (rep > 0) best = std::min(best, t);  // the first run warms up
        }
        *ms = best;
        return HN_OK;
    };
    hn_tune_result r{};
    r.n_sizes = n_sizes;
    hn_status st = HN_OK;
    const bool dense_ok = dense_scan_supported(ix);
    int32_t dense_min = 0x7FFFFFFF;
    std::vector<int64_t> order(sizes, sizes + n_sizes);
    for (int32_t i = 0; st == HN_OK && i < n_sizes; ++i) {
        r.sizes[i] = sizes[i];
        st = time_search(sizes[i], HN_SCAN_STREAM, &r.ms_stream[i]);
        r.ms_dense[i] = -1.f;
        if (st == HN_OK && dense_ok) st = time_search(sizes[i], HN_SCAN_DENSE, &r.ms_dense[i]);
    }
    if (st == HN_OK && dense_ok) {
        // smallest tuned size from which the dense scan wins at every larger tuned size
        std::vector<int32_t> idx(n_sizes);
        for (int32_t i = 0; i < n_sizes; ++i) idx[i] = i;
        std::sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) { return r.sizes[x] < r.sizes[y]; });
        for (int32_t j = n_sizes - 1; j >= 0 && r.ms_dense[idx[j]] <= r.ms_stream[idx[j]]; --j)
            dense_min = (int32_t)std::min<int64_t>(r.sizes[idx[j]], 0x7FFFFFFF);
        ix.dense_min_q = dense_min;
        // dense work-unit granularity at the largest tuned size
        if (dense_min != 0x7FFFFFFF) {
            float bt = 1e30f;
            int32_t bu = ix.units_per_cta;
            const int32_t cand[4] = {32, 64, 128, 256};
            for (int c = 0; st == HN_OK && c < 4; ++c) {
                ix.units_per_cta = cand[c];
                float t = 0;
                st = time_search(qmax, HN_SCAN_DENSE, &t);
                r.ms_units[c] = t;
                if (t < bt) { bt = t; bu = cand[c]; }
            }
            ix.units_per_cta = bu;
        }
    }
    r.dense_min_q = ix.dense_min_q;
    r.units_per_cta = ix.units_per_cta;
    cudaFree(oi);
    cudaFree(os);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != HN_OK) return st;
    if (out) *out = r;
    return HN_OK;
}

}  // extern "C"
