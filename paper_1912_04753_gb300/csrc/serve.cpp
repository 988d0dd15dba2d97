// Serving loop: resident point sets, worker slots with their own streams, admission by device
// memory and continuous batching of compatible jobs (the GPU counterpart of the paper's
// job-submission tier, Section 5).
//
// Scheduling, all under one mutex:
//   queue   - submitted jobs in arrival order;
//   slots   - a worker takes the first queued job whose point set is idle, plus every later
//             queued job on that point set with identical thresholds and modes (the batch);
//   memory  - accounted = point sets + grants of running batches + workspaces that idle point
//             sets still hold.  A batch needs at least fixed + per_real bytes (one realization
//             per wave); the worker releases idle workspaces (least recently used first) until
//             that fits, waits for running batches otherwise, and fails the batch with
//             STK_ENOMEM only when nothing else holds memory.  The grant is then as much of
//             the whole batch as fits, and the job runner sizes its waves to it.
// Determinism: realization k of a job is Philox realization k under the job's seed whatever
// the batch, and every realization is accumulated in its own exact fixed-point histogram, so a
// job's grids are the same alone and merged.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "stk.h"
#include "stk_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

int note(int code, const char* msg) {
    stk::stk_note_error(code, msg);
    return code;
}

enum class JobState { Queued, Running, Done, Failed };

struct Job {
    uint64_t ticket = 0;
    uint64_t dataset = 0;
    std::vector<double> s, tt;
    int edge_mode = 0, prec = 0, norm = 0, n_sims = 0, want_sims = 0, sim_method = 0;
    int n_sectors = 0;
    uint64_t seed = 0;
    JobState state = JobState::Queued;
    int rc = STK_OK;
    std::string err;
    Clock::time_point t_submit, t_done;
    // results
    std::vector<double> K, L, S, env, K_sims;
    std::vector<int64_t> C, C_sims;
};

struct Dataset {
    stk_handle* h = nullptr;
    int64_t n = 0;
    size_t point_bytes = 0;
    bool busy = false;
    size_t idle_bytes = 0;  // workspace held while idle (accounted)
    uint64_t last_used = 0;
    int pending = 0;        // queued + running jobs
};

// The request of a batch headed by `head` (thresholds, modes; n_sims and seeds come from the
// batch's plan).
stk_request head_request(const Job& head) {
    stk_request q;
    memset(&q, 0, sizeof q);
    q.s = head.s.data();
    q.cs = (int)head.s.size();
    q.tt = head.tt.data();
    q.ct = (int)head.tt.size();
    q.edge_mode = head.edge_mode;
    q.prec = head.prec;
    q.norm = head.norm;
    q.exec = STK_EXEC_BATCHED;
    q.sim_method = head.sim_method;
    q.n_sectors = head.n_sectors;
    return q;
}

bool same_params(const Job& a, const Job& b) {
    return a.dataset == b.dataset && a.s == b.s && a.tt == b.tt && a.edge_mode == b.edge_mode &&
           a.prec == b.prec && a.norm == b.norm && a.sim_method == b.sim_method &&
           a.n_sectors == b.n_sectors;
}

}  // namespace

struct stk_server {
    stk_server_config cfg{};
    size_t budget = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::vector<std::thread> workers;
    std::map<uint64_t, Dataset> datasets;
    std::map<uint64_t, std::shared_ptr<Job>> jobs;
    std::deque<uint64_t> queue;
    uint64_t next_ticket = 1, next_dataset = 1, use_clock = 0;
    size_t points_total = 0, granted = 0, idle_total = 0, peak = 0;
    int running = 0;
    // statistics since the last reset
    int64_t submitted = 0, completed = 0, failed = 0, max_depth = 0, batches = 0, merged = 0;
    int64_t sims_done = 0, pairs = 0, launches = 0, fused_jobs = 0;
    std::vector<double> lat_ms;
    bool have_first = false;
    Clock::time_point t_first, t_last;

    size_t accounted() const { return points_total + granted + idle_total; }
    void note_peak() { peak = std::max(peak, accounted()); }
};

namespace {

// Releases idle workspaces (least recently used first, never `keep`) until `need` bytes are
// free under the budget.  Called with the lock held; the handles involved are idle.
void release_idle(stk_server* sv, size_t need, uint64_t keep) {
    while (sv->accounted() + need > sv->budget) {
        Dataset* victim = nullptr;
        for (auto& kv : sv->datasets) {
            Dataset& d = kv.second;
            if (kv.first == keep || d.busy || d.idle_bytes == 0) continue;
            if (!victim || d.last_used < victim->last_used) victim = &d;
        }
        if (!victim) return;
        stk::handle_trim(victim->h);
        sv->idle_total -= victim->idle_bytes;
        victim->idle_bytes = 0;
    }
}

struct Batch {
    uint64_t dataset = 0;
    std::vector<std::shared_ptr<Job>> jobs;
    size_t grant = 0;
};

// A fused group being formed: its point sets and the point-realizations it may still take.
struct FuseGroup {
    std::vector<uint64_t> datasets;
    double room = 0.0;
};

// Picks the next batch and admits it (lock held).  Returns false when nothing can start now.
// fuse: a fused group being formed; then only a batch on another point set that can share the
// group's pair launch (a small job that fits one wave now and the group's room) is taken, and
// nothing is failed or waited for.
bool take_batch(stk_server* sv, Batch* out, FuseGroup* fuse = nullptr) {
    for (size_t qi = 0; qi < sv->queue.size(); ++qi) {
        auto jt = sv->jobs.find(sv->queue[qi]);
        if (jt == sv->jobs.end()) continue;
        std::shared_ptr<Job> head = jt->second;
        Dataset& ds = sv->datasets[head->dataset];
        if (ds.busy) continue;
        if (fuse) {
            if (std::find(fuse->datasets.begin(), fuse->datasets.end(), head->dataset) !=
                fuse->datasets.end())
                continue;
            const stk_request hq = head_request(*head);
            if (!stk::fusable_job(ds.h, &hq, 1 + (int64_t)head->n_sims) ||
                (double)ds.n * (1.0 + head->n_sims) > fuse->room)
                continue;
        }
        // the batch: the head plus compatible queued jobs, in arrival order
        std::vector<size_t> take{qi};
        int sims = head->n_sims;
        const int cap = sv->cfg.max_batch_sims;
        if (!sv->cfg.no_merge) {
            for (size_t k = qi + 1; k < sv->queue.size(); ++k) {
                auto it = sv->jobs.find(sv->queue[k]);
                if (it == sv->jobs.end()) continue;
                const Job& j = *it->second;
                if (!same_params(*head, j) || sims + j.n_sims > cap) continue;
                sims += j.n_sims;
                take.push_back(k);
            }
        }
        int groups = 0;
        for (size_t k : take) groups += sv->jobs[sv->queue[k]]->n_sims > 0 ? 1 : 0;
        const stk_request q = head_request(*head);
        stk::Footprint fp;
        const int R = 1 + sims;
        int rc = stk::job_footprint(ds.h, &q, R, groups, &fp);
        if (rc == STK_OK) {
            const size_t need_min = fp.fixed + fp.per_real;
            // this point set's own idle workspace is reused by the batch
            const size_t own = ds.idle_bytes;
            sv->idle_total -= own;
            ds.idle_bytes = 0;
            release_idle(sv, std::max(need_min, own), head->dataset);
            if (sv->accounted() + need_min > sv->budget && own > 0) {
                stk::handle_trim(ds.h);  // the old workspace does not fit beside the minimum
                release_idle(sv, need_min, head->dataset);
            }
            const size_t free_now =
                sv->budget > sv->accounted() ? sv->budget - sv->accounted() : 0;
            if (stk::handle_workspace_bytes(ds.h) > free_now) stk::handle_trim(ds.h);
            if (fuse && ((double)ds.n * R > fuse->room ||
                         fp.fixed + fp.per_real * (size_t)R > free_now)) {
                const size_t still = stk::handle_workspace_bytes(ds.h);
                sv->idle_total += still;  // not now: it would not run in one wave
                ds.idle_bytes = still;
                continue;
            }
            if (need_min > free_now) {
                const size_t still = stk::handle_workspace_bytes(ds.h);
                sv->idle_total += still;
                ds.idle_bytes = still;
                if (sv->running > 0) return false;  // wait for memory (arrival order kept)
                rc = STK_ENOMEM;
                char buf[200];
                snprintf(buf, sizeof buf,
                         "job needs %zu bytes of device memory at least; the server budget "
                         "leaves %zu",
                         need_min, free_now);
                head->err = buf;
            } else {
                const size_t whole = fp.fixed + fp.per_real * (size_t)R;
                out->grant = std::max(std::min(whole, free_now), stk::handle_workspace_bytes(ds.h));
            }
        } else {
            head->err = stk_last_error();
        }
        if (rc != STK_OK) {  // fail the head job only
            head->state = JobState::Failed;
            head->rc = rc;
            head->t_done = Clock::now();
            sv->queue.erase(sv->queue.begin() + (long)qi);
            ds.pending -= 1;
            sv->failed += 1;
            sv->cv_done.notify_all();
            --qi;
            continue;
        }
        out->dataset = head->dataset;
        out->jobs.clear();
        for (size_t k : take) out->jobs.push_back(sv->jobs[sv->queue[k]]);
        for (size_t k = take.size(); k-- > 0;) sv->queue.erase(sv->queue.begin() + (long)take[k]);
        for (auto& j : out->jobs) j->state = JobState::Running;
        ds.busy = true;
        ds.last_used = ++sv->use_clock;
        sv->granted += out->grant;
        sv->running += 1;
        sv->note_peak();
        return true;
    }
    return false;
}

// A batch's request and simulation plan: every job's simulations under its own seed, its
// envelope group and first row.
struct BatchRun {
    stk_request q;
    stk::SimPlan plan;
    std::vector<int> group_of, first_row;
    bool any_sims = false;
};

void plan_batch(const Batch& b, BatchRun* br) {
    br->q = head_request(*b.jobs[0]);
    stk::SimPlan& plan = br->plan;
    std::vector<int>& group_of = br->group_of;
    std::vector<int>& first_row = br->first_row;
    group_of.assign(b.jobs.size(), -1);
    first_row.assign(b.jobs.size(), 0);
    bool any_sims = false;
    for (size_t j = 0; j < b.jobs.size(); ++j) {
        const Job& job = *b.jobs[j];
        first_row[j] = 1 + (int)plan.seed.size();
        if (job.n_sims > 0) {
            group_of[j] = (int)plan.groups.size();
            plan.groups.push_back({(int)plan.seed.size(), job.n_sims});
            for (int k = 0; k < job.n_sims; ++k) {
                plan.seed.push_back(job.seed);
                plan.id.push_back((uint32_t)k);
            }
            any_sims = any_sims || job.want_sims;
        }
    }
    br->any_sims = any_sims;
}

// Copies the batch's results (the last job run on h) into its jobs.
int collect_batch(stk_handle* h, Batch& b, const BatchRun& br, int64_t* qual,
                  int64_t* launches) {
    const stk_request& q = br.q;
    const stk::SimPlan& plan = br.plan;
    const std::vector<int>& group_of = br.group_of;
    const std::vector<int>& first_row = br.first_row;
    const bool any_sims = br.any_sims;
    int rc = STK_OK;
    const int nbins = q.cs * q.ct * (q.n_sectors > 1 ? q.n_sectors : 1);
    const int R = 1 + (int)plan.seed.size();
    std::vector<double> K(nbins), L(nbins), S(nbins), env(4 * (size_t)nbins * plan.groups.size());
    std::vector<int64_t> C(nbins);
    std::vector<double> Ks;
    std::vector<int64_t> Cs;
    if ((rc = stk::fetch_rows(h, 0, 0, 1, K.data())) || (rc = stk::fetch_rows(h, 1, 0, 1, L.data())) ||
        (rc = stk::fetch_rows(h, 2, 0, 1, S.data())) || (rc = stk::fetch_rows(h, 3, 0, 1, C.data())))
        return rc;
    if (!plan.groups.empty() &&
        (rc = stk::fetch_rows(h, 4, 0, 4 * (int)plan.groups.size(), env.data())))
        return rc;
    if (any_sims) {
        Ks.resize((size_t)(R - 1) * nbins);
        Cs.resize((size_t)(R - 1) * nbins);
        if ((rc = stk::fetch_rows(h, 0, 1, R - 1, Ks.data())) ||
            (rc = stk::fetch_rows(h, 3, 1, R - 1, Cs.data())))
            return rc;
    }
    if ((rc = stk::handle_sync(h))) return rc;
    stk_stats st;
    stk_last_stats(h, &st);
    *qual = st.qualifying_pairs;
    *launches = st.kernel_launches;
    for (size_t j = 0; j < b.jobs.size(); ++j) {
        Job& job = *b.jobs[j];
        job.K = K;
        job.L = L;
        job.S = S;
        job.C = C;
        if (group_of[j] >= 0) {
            const size_t o = (size_t)group_of[j] * 4 * nbins;
            job.env.assign(env.begin() + (long)o, env.begin() + (long)(o + 4 * (size_t)nbins));
            if (job.want_sims) {
                const size_t r0 = (size_t)(first_row[j] - 1) * nbins;
                const size_t len = (size_t)job.n_sims * nbins;
                job.K_sims.assign(Ks.begin() + (long)r0, Ks.begin() + (long)(r0 + len));
                job.C_sims.assign(Cs.begin() + (long)r0, Cs.begin() + (long)(r0 + len));
            }
        }
    }
    return STK_OK;
}

// Runs one batch on its point set's stream (lock not held).  Fills the jobs' results.
int run_batch(stk_handle* h, Batch& b, int64_t* qual, int64_t* launches) {
    BatchRun br;
    plan_batch(b, &br);
    stk::handle_set_wave_budget(h, b.grant);
    const int rc = stk::run_plan(h, &br.q, br.plan, true);
    if (rc) return rc;
    return collect_batch(h, b, br, qual, launches);
}

// Runs batches on different point sets with their pair kernels in shared launches (lock not
// held); per batch its status, qualifying pairs and kernel launches.
void run_fused_group(std::vector<Batch>& group, const std::vector<stk_handle*>& hs,
                     std::vector<int>* rcs, std::vector<int64_t>* quals,
                     std::vector<int64_t>* launches) {
    const size_t ng = group.size();
    std::vector<BatchRun> brs(ng);
    std::vector<stk::FusePart> parts;
    for (size_t i = 0; i < ng; ++i) {
        plan_batch(group[i], &brs[i]);
        stk::handle_set_wave_budget(hs[i], group[i].grant);
        parts.push_back({hs[i], &brs[i].q, &brs[i].plan});
    }
    int fused = 0;
    const int rc = stk::run_plans_fused(parts, &fused);
    rcs->assign(ng, rc);
    quals->assign(ng, 0);
    launches->assign(ng, 0);
    if (rc) return;
    for (size_t i = 0; i < ng; ++i)
        (*rcs)[i] = collect_batch(hs[i], group[i], brs[i], &(*quals)[i], &(*launches)[i]);
}

// Bookkeeping after a batch ran (lock held).
void finish_batch(stk_server* sv, Batch& b, int rc, const std::string& err, int64_t qual,
                  int64_t launches, Clock::time_point now) {
    stk_handle* h = sv->datasets[b.dataset].h;
    sv->granted -= b.grant;
    sv->running -= 1;
    Dataset& d2 = sv->datasets[b.dataset];
    d2.busy = false;
    d2.pending -= (int)b.jobs.size();
    d2.idle_bytes = stk::handle_workspace_bytes(h);
    sv->idle_total += d2.idle_bytes;
    if (sv->accounted() > sv->budget) {  // the runner held more than granted: give it back
        sv->idle_total -= d2.idle_bytes;
        stk::handle_trim(h);
        d2.idle_bytes = 0;
    }
    sv->batches += 1;
    if (b.jobs.size() > 1) sv->merged += (int64_t)b.jobs.size();
    if (rc == STK_OK) sv->pairs += qual;
    sv->launches += launches;
    for (auto& jp : b.jobs) {
        Job& j = *jp;
        j.t_done = now;
        if (rc == STK_OK) {
            j.state = JobState::Done;
            sv->completed += 1;
            sv->sims_done += j.n_sims;
            sv->lat_ms.push_back(
                std::chrono::duration<double, std::milli>(now - j.t_submit).count());
            sv->t_last = now;
        } else {
            j.state = JobState::Failed;
            j.rc = rc;
            j.err = err;
            sv->failed += 1;
        }
    }
}

constexpr size_t kMaxFusedBatches = 16;

void worker_main(stk_server* sv) {
    cudaSetDevice(sv->cfg.device);
    std::unique_lock<std::mutex> lock(sv->mu);
    while (!sv->stop) {
        std::vector<Batch> group(1);
        if (!take_batch(sv, &group[0])) {
            sv->cv_work.wait(lock);
            continue;
        }
        // a small batch takes the next small batches on other idle point sets into its launch
        if (sv->cfg.fuse) {
            int sims = 0;
            for (const auto& j : group[0].jobs) sims += j->n_sims;
            const stk_request hq = head_request(*group[0].jobs[0]);
            const Dataset& d0 = sv->datasets[group[0].dataset];
            if (stk::fusable_job(d0.h, &hq, 1 + (int64_t)sims)) {
                // a group holds about as much work as one job that is just too large to fuse,
                // so that fusing gathers small jobs without starving the other slots
                FuseGroup fg;
                fg.datasets.push_back(group[0].dataset);
                fg.room = stk::kFuseMaxPointRealizations - (double)d0.n * (1.0 + sims);
                while (group.size() < kMaxFusedBatches) {
                    Batch bk;
                    if (!take_batch(sv, &bk, &fg)) break;
                    int bs = 0;
                    for (const auto& j : bk.jobs) bs += j->n_sims;
                    fg.datasets.push_back(bk.dataset);
                    fg.room -= (double)sv->datasets[bk.dataset].n * (1.0 + bs);
                    group.push_back(std::move(bk));
                }
            }
        }
        std::vector<stk_handle*> hs;
        for (const Batch& b : group) hs.push_back(sv->datasets[b.dataset].h);
        lock.unlock();
        std::vector<int> rcs;
        std::vector<int64_t> quals, launches;
        if (group.size() == 1) {
            int64_t qual = 0, nl = 0;
            rcs.push_back(run_batch(hs[0], group[0], &qual, &nl));
            quals.push_back(qual);
            launches.push_back(nl);
        } else {
            run_fused_group(group, hs, &rcs, &quals, &launches);
        }
        std::string err;
        for (int rc : rcs)
            if (rc) err = stk_last_error();
        const auto now = Clock::now();
        lock.lock();
        for (size_t i = 0; i < group.size(); ++i) {
            finish_batch(sv, group[i], rcs[i], err, quals[i], launches[i], now);
            if (group.size() > 1) sv->fused_jobs += (int64_t)group[i].jobs.size();
        }
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
}

double percentile(std::vector<double> v, double p) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    // nearest-rank percentile
    size_t k = (size_t)std::ceil(p / 100.0 * (double)v.size());
    if (k < 1) k = 1;
    if (k > v.size()) k = v.size();
    return v[k - 1];
}

}  // namespace

extern "C" {

int stk_server_create(const stk_server_config* cfg, stk_server** out) {
    if (!cfg || !out) return note(STK_EINVAL, "config and out must not be NULL");
    *out = nullptr;
    if (cfg->slots < 0 || cfg->slots > 64) return note(STK_EINVAL, "slots must be in [0, 64]");
    if (cfg->mem_budget_bytes < 0 || cfg->max_batch_sims < 0 || cfg->max_queue < 0)
        return note(STK_EINVAL, "negative server limit");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return note(STK_ENODEV, "no CUDA device");
    }
    if (cfg->device < 0 || cfg->device >= ndev) return note(STK_EINVAL, "no such device");
    if (cudaSetDevice(cfg->device) != cudaSuccess) {
        cudaGetLastError();
        return note(STK_ECUDA, "cudaSetDevice failed");
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return note(STK_ECUDA, "cudaMemGetInfo failed");
    }
    stk_server* sv = new stk_server();
    sv->cfg = *cfg;
    if (sv->cfg.slots == 0) sv->cfg.slots = 4;
    if (sv->cfg.max_batch_sims == 0) sv->cfg.max_batch_sims = 8192;
    if (sv->cfg.max_queue == 0) sv->cfg.max_queue = 65536;
    sv->budget = cfg->mem_budget_bytes ? (size_t)cfg->mem_budget_bytes
                                       : (size_t)(0.8 * (double)free_b);
    for (int k = 0; k < sv->cfg.slots; ++k) sv->workers.emplace_back(worker_main, sv);
    *out = sv;
    return STK_OK;
}

int stk_server_register(stk_server* sv, const double* x, const double* y, const double* t,
                        int64_t n, const stk_box* box, uint64_t* dataset) {
    if (!sv || !dataset) return note(STK_EINVAL, "server and dataset must not be NULL");
    const size_t bytes = 24 * (size_t)(n > 0 ? n : 0);
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        release_idle(sv, bytes, 0);
        if (sv->accounted() + bytes > sv->budget)
            return note(STK_ENOMEM, "point set does not fit the server's memory budget");
        sv->points_total += bytes;  // reserved while the copy runs
        sv->note_peak();
    }
    cudaSetDevice(sv->cfg.device);
    stk_handle* h = nullptr;
    const int rc = stk_create(x, y, t, n, box, &h);
    std::lock_guard<std::mutex> lock(sv->mu);
    if (rc) {
        sv->points_total -= bytes;
        return rc;
    }
    const uint64_t id = sv->next_dataset++;
    Dataset& d = sv->datasets[id];
    d.h = h;
    d.n = n;
    d.point_bytes = bytes;
    *dataset = id;
    return STK_OK;
}

int stk_server_unregister(stk_server* sv, uint64_t dataset) {
    if (!sv) return note(STK_EINVAL, "server is NULL");
    stk_handle* h = nullptr;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        auto it = sv->datasets.find(dataset);
        if (it == sv->datasets.end()) return note(STK_EINVAL, "unknown dataset");
        if (it->second.busy || it->second.pending > 0)
            return note(STK_EBUSY, "jobs on this dataset are queued or running");
        h = it->second.h;
        sv->points_total -= it->second.point_bytes;
        sv->idle_total -= it->second.idle_bytes;
        sv->datasets.erase(it);
    }
    stk_destroy(h);
    return STK_OK;
}

}  // extern "C"

namespace {

// Applies `fn` to an idle point set's handle outside the server lock (the point set is marked
// busy meanwhile, so no batch starts on it); STK_EBUSY while jobs on it are queued or running.
template <class F>
int with_idle_dataset(stk_server* sv, uint64_t dataset, F fn) {
    stk_handle* h = nullptr;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        auto it = sv->datasets.find(dataset);
        if (it == sv->datasets.end()) return note(STK_EINVAL, "unknown dataset");
        if (it->second.busy || it->second.pending > 0)
            return note(STK_EBUSY, "jobs on this dataset are queued or running");
        it->second.busy = true;
        h = it->second.h;
    }
    const int rc = fn(h);
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->datasets[dataset].busy = false;
    }
    sv->cv_work.notify_all();
    return rc;
}

}  // namespace

extern "C" {

int stk_server_set_polygon(stk_server* sv, uint64_t dataset, const double* vx, const double* vy,
                           int nv) {
    if (!sv) return note(STK_EINVAL, "server is NULL");
    return with_idle_dataset(sv, dataset,
                             [&](stk_handle* h) { return stk_set_polygon(h, vx, vy, nv); });
}

int stk_server_set_intensity(stk_server* sv, uint64_t dataset, const double* rho, int nix,
                             int niy, int nit) {
    if (!sv) return note(STK_EINVAL, "server is NULL");
    return with_idle_dataset(
        sv, dataset, [&](stk_handle* h) { return stk_set_intensity(h, rho, nix, niy, nit); });
}

int stk_submit(stk_server* sv, const stk_job* job, uint64_t* ticket) {
    if (!sv || !job || !ticket) return note(STK_EINVAL, "server, job and ticket must not be NULL");
    if (!job->s || !job->tt || job->cs < 1 || job->ct < 1 || job->cs > STK_MAX_THRESHOLDS ||
        job->ct > STK_MAX_THRESHOLDS)
        return note(STK_EINVAL, "threshold arrays must hold 1..64 entries");
    if (job->n_sims < 0 || job->n_sims > (1 << 20)) return note(STK_EINVAL, "n_sims out of range");
    if (job->edge_mode != STK_EDGE_NONE && job->edge_mode != STK_EDGE_ISOTROPIC &&
        job->edge_mode != STK_EDGE_TRANSLATION)
        return note(STK_EINVAL, "unknown edge_mode");
    if (job->prec != STK_PREC_FP64 && job->prec != STK_PREC_FP32_GUARDED)
        return note(STK_EINVAL, "unknown prec");
    if (job->norm != STK_NORM_N_NM1 && job->norm != STK_NORM_N2)
        return note(STK_EINVAL, "unknown norm");
    if (job->sim_method < STK_SIM_CSR || job->sim_method > STK_SIM_BOOTSTRAP)
        return note(STK_EINVAL, "unknown sim_method");
    if (job->n_sectors < 0 || job->n_sectors > 64 ||
        (job->n_sectors > 1 && job->n_sectors * job->cs * job->ct > 4096))
        return note(STK_EINVAL, "n_sectors out of range (n_sectors * cs * ct <= 4096)");
    auto j = std::make_shared<Job>();
    j->dataset = job->dataset;
    j->s.assign(job->s, job->s + job->cs);
    j->tt.assign(job->tt, job->tt + job->ct);
    j->edge_mode = job->edge_mode;
    j->prec = job->prec;
    j->norm = job->norm;
    j->n_sims = job->n_sims;
    j->seed = job->seed;
    j->want_sims = job->want_sims;
    j->sim_method = job->sim_method;
    j->n_sectors = job->n_sectors;
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->datasets.find(job->dataset);
    if (it == sv->datasets.end()) return note(STK_EINVAL, "unknown dataset");
    {
        // thresholds checked against the point set's box now, not when the job runs
        stk::Footprint fp;
        stk_request q;
        memset(&q, 0, sizeof q);
        q.s = j->s.data();
        q.cs = job->cs;
        q.tt = j->tt.data();
        q.ct = job->ct;
        q.edge_mode = job->edge_mode;
        q.n_sectors = job->n_sectors;
        const int rc = stk::job_footprint(it->second.h, &q, 1, 0, &fp);
        if (rc) return rc;
    }
    if ((int)sv->queue.size() >= sv->cfg.max_queue) return note(STK_EBUSY, "queue full");
    j->ticket = sv->next_ticket++;
    j->t_submit = Clock::now();
    if (!sv->have_first) {
        sv->have_first = true;
        sv->t_first = j->t_submit;
    }
    sv->jobs[j->ticket] = j;
    sv->queue.push_back(j->ticket);
    it->second.pending += 1;
    sv->submitted += 1;
    sv->max_depth = std::max<int64_t>(sv->max_depth, (int64_t)sv->queue.size());
    *ticket = j->ticket;
    sv->cv_work.notify_one();
    return STK_OK;
}

int stk_poll(stk_server* sv, uint64_t ticket, stk_result* res, int wait_ms, double* latency_ms) {
    if (!sv) return note(STK_EINVAL, "server is NULL");
    std::shared_ptr<Job> j;
    {
        std::unique_lock<std::mutex> lock(sv->mu);
        auto it = sv->jobs.find(ticket);
        if (it == sv->jobs.end()) return note(STK_EINVAL, "unknown ticket");
        j = it->second;
        auto finished = [&] { return j->state == JobState::Done || j->state == JobState::Failed; };
        if (wait_ms < 0)
            sv->cv_done.wait(lock, finished);
        else if (!sv->cv_done.wait_for(lock, std::chrono::milliseconds(wait_ms), finished))
            return note(STK_ETIMEOUT, "job not finished yet");
        sv->jobs.erase(ticket);
    }
    if (latency_ms)
        *latency_ms = std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count();
    if (j->state == JobState::Failed) return note(j->rc, j->err.c_str());
    if (res) {
        const size_t nb = j->K.size();
        auto put = [nb](void* dst, const void* src, size_t elt) {
            if (dst) memcpy(dst, src, nb * elt);
        };
        put(res->K, j->K.data(), 8);
        put(res->L, j->L.data(), 8);
        put(res->raw_sum, j->S.data(), 8);
        put(res->pair_count, j->C.data(), 8);
        if (j->n_sims > 0) {
            put(res->K_lo, j->env.data(), 8);
            put(res->K_hi, j->env.data() + nb, 8);
            put(res->L_lo, j->env.data() + 2 * nb, 8);
            put(res->L_hi, j->env.data() + 3 * nb, 8);
            if (res->K_sims || res->count_sims) {
                if (!j->want_sims) return note(STK_EINVAL, "per-realization grids need want_sims");
                if (res->K_sims) memcpy(res->K_sims, j->K_sims.data(), 8 * j->K_sims.size());
                if (res->count_sims)
                    memcpy(res->count_sims, j->C_sims.data(), 8 * j->C_sims.size());
            }
        }
    }
    return STK_OK;
}

int stk_server_stats(stk_server* sv, stk_serve_stats* out) {
    if (!sv || !out) return note(STK_EINVAL, "server and out must not be NULL");
    std::lock_guard<std::mutex> lock(sv->mu);
    memset(out, 0, sizeof *out);
    out->submitted = sv->submitted;
    out->completed = sv->completed;
    out->failed = sv->failed;
    out->queued = (int64_t)sv->queue.size();
    out->running = sv->running;
    out->max_queue_depth = sv->max_depth;
    out->batches = sv->batches;
    out->merged_jobs = sv->merged;
    out->simulations = sv->sims_done;
    out->qualifying_pairs = sv->pairs;
    out->kernel_launches = sv->launches;
    out->fused_jobs = sv->fused_jobs;
    out->p50_ms = percentile(sv->lat_ms, 50.0);
    out->p99_ms = percentile(sv->lat_ms, 99.0);
    double mx = 0, sum = 0;
    for (double v : sv->lat_ms) mx = std::max(mx, v), sum += v;
    out->max_ms = mx;
    out->mean_ms = sv->lat_ms.empty() ? 0.0 : sum / (double)sv->lat_ms.size();
    if (sv->have_first && sv->completed > 0) {
        out->wall_s = std::chrono::duration<double>(sv->t_last - sv->t_first).count();
        if (out->wall_s > 0) {
            out->jobs_per_s = (double)sv->completed / out->wall_s;
            out->sims_per_s = (double)sv->sims_done / out->wall_s;
        }
    }
    out->resident_bytes = (int64_t)sv->accounted();
    out->peak_bytes = (int64_t)sv->peak;
    out->budget_bytes = (int64_t)sv->budget;
    return STK_OK;
}

int stk_server_reset_stats(stk_server* sv) {
    if (!sv) return note(STK_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->submitted = sv->completed = sv->failed = sv->max_depth = 0;
    sv->batches = sv->merged = sv->sims_done = sv->pairs = sv->launches = sv->fused_jobs = 0;
    sv->lat_ms.clear();
    sv->have_first = false;
    sv->peak = sv->accounted();
    return STK_OK;
}

void stk_server_destroy(stk_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
        for (uint64_t t : sv->queue) {
            auto it = sv->jobs.find(t);
            if (it == sv->jobs.end()) continue;
            it->second->state = JobState::Failed;
            it->second->rc = STK_EBUSY;
            it->second->err = "server shut down before the job ran";
        }
        sv->queue.clear();
    }
    sv->cv_work.notify_all();
    sv->cv_done.notify_all();
    for (auto& w : sv->workers) w.join();
    for (auto& kv : sv->datasets) stk_destroy(kv.second.h);
    delete sv;
}

}  // extern "C"
