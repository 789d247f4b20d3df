// Served classification (mc_server, include/mc.h): a resident database, a
// job queue and a scheduler thread that admits jobs by device memory and
// packs them into launch sets of a classification plan (continuous
// batching).  Host code only; every step of the method runs in the kernels
// behind mc_plan_run and mc_db_add_targets / mc_db_finalize.
//
// Threads and locking.  Callers (submit, extend, wait, stats) and the CUDA
// host callbacks that report finished launch sets only touch the shared
// state under `mu`; the scheduler thread takes `mu` to read and update that
// state but never holds it across a CUDA call, so a host callback is never
// blocked by a thread that is itself waiting for the GPU.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mc.h"

namespace mc {
// Records the message of mc_last_error_string and returns `code` (mc_api.cu).
int report_error(int code, const char* fmt, ...);
}

namespace {

using Clock = std::chrono::steady_clock;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Job {
    uint64_t id = 0;
    mc_job j{};
    double t_submit = 0, t_launch = -1, t_done = 0;
    uint64_t epoch = 0;
    uint32_t pieces = 0, pieces_left = 0;
    uint32_t next_q = 0;  // first query not yet in a launch set
    uint64_t ext_seq = 0;  // extensions requested before the job: it runs after they are applied
    int status = MC_OK;
    bool done = false;
    // device copy: seq | offs | qoffs | label | hits | top
    unsigned char* dbuf = nullptr;
    size_t bytes = 0;
    size_t o_offs = 0, o_qoffs = 0, o_label = 0, o_hits = 0, o_top = 0;
    cudaEvent_t copied = nullptr;
};

struct Extension {
    std::vector<char> seq;
    std::vector<uint64_t> offs;
    std::vector<uint32_t> taxon;
};

struct Piece {
    Job* job;
    uint32_t q0, q1;
};

struct Slot;

struct CallbackCtx {
    mc_server* srv;
    int slot;
};

struct Slot {
    cudaStream_t stream = nullptr;
    mc_plan* plan = nullptr;
    bool busy = false;
    std::vector<Piece> pieces;
    CallbackCtx ctx{};
};

size_t job_bytes(const mc_job& j, size_t* o_offs, size_t* o_qoffs, size_t* o_label, size_t* o_hits, size_t* o_top) {
    const uint64_t seq_bytes = j.n_seq ? j.offs[j.n_seq] : 0;
    size_t o = align256(seq_bytes + 16);
    *o_offs = o;
    o = align256(o + ((size_t)j.n_seq + 1) * 8);
    *o_qoffs = o;
    o = align256(o + ((size_t)j.n_queries + 1) * 4);
    *o_label = o;
    o = align256(o + (size_t)j.n_queries * 4);
    *o_hits = o;
    o = align256(o + (size_t)j.n_queries * 4);
    *o_top = o;
    o = align256(o + (size_t)j.n_queries * 4);
    return o;
}

}  // namespace

struct mc_server {
    mc_db* db = nullptr;
    mc_classify_params params{};
    uint32_t max_set_queries = 0, max_set_jobs = 0;
    uint64_t hbm_limit = 0;
    Clock::time_point t0;
    std::vector<Slot> slots;
    cudaStream_t copy_stream = nullptr;
    int device = 0;

    std::mutex mu;
    std::condition_variable cv;       // scheduler wake-up
    std::condition_variable done_cv;  // job completions, drain
    uint64_t events = 0;              // bumped by every submit / extend / completion / stop
    bool stop = false;
    uint64_t next_id = 1;
    std::unordered_map<uint64_t, std::unique_ptr<Job>> jobs;
    std::deque<Job*> arrivals;        // submitted, not admitted
    std::deque<Job*> admitted;        // device copy made, queries left to launch
    std::deque<Extension> extensions;
    std::vector<int> completed;       // slots whose launch set finished
    std::vector<double> completed_t;
    uint64_t in_flight = 0;           // busy slots
    bool working = false;             // the scheduler holds work taken from the queues
    // statistics
    uint64_t jobs_submitted = 0, jobs_done = 0, queries_done = 0, launch_sets = 0, n_ext = 0, epoch = 0;
    uint64_t ext_requested = 0, ext_applied = 0;
    std::vector<double> ext_seconds;  // time of each applied extension (add + finalize)
    uint64_t hbm_in_use = 0, hbm_peak = 0;
    double t_first = -1, t_last = 0;
    std::vector<double> latencies;
    uint32_t next_target = 0;

    std::thread th;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
    void run();
    bool idle_locked() const {
        return arrivals.empty() && admitted.empty() && extensions.empty() && in_flight == 0 && completed.empty() &&
               !working;
    }
};

namespace {

void CUDART_CB on_set_done(void* p) {
    auto* c = static_cast<CallbackCtx*>(p);
    mc_server* s = c->srv;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->completed.push_back(c->slot);
        s->completed_t.push_back(s->now());
        ++s->events;
    }
    s->cv.notify_one();
}

// Applies one extension: device copy, add, finalize (synchronous).
int apply_extension(mc_server* s, Extension& e, uint64_t* epoch_out) {
    const uint32_t n = (uint32_t)e.taxon.size();
    void* dseq = nullptr;
    void* doffs = nullptr;
    cudaStream_t cs = s->copy_stream;
    const size_t sb = std::max<size_t>(e.seq.size(), 1);
    if (cudaMallocAsync(&dseq, sb, cs) != cudaSuccess || cudaMallocAsync(&doffs, e.offs.size() * 8, cs) != cudaSuccess) {
        cudaGetLastError();
        if (dseq) cudaFreeAsync(dseq, cs);
        return MC_ERR_OOM;
    }
    int rc = MC_OK;
    // pageable sources: each copy is staged before the call returns
    if (cudaMemcpyAsync(dseq, e.seq.data(), e.seq.size(), cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaMemcpyAsync(doffs, e.offs.data(), e.offs.size() * 8, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaStreamSynchronize(cs) != cudaSuccess) {
        cudaGetLastError();
        rc = MC_ERR_CUDA;
    }
    // add + finalize run on the database stream and return after it is idle;
    // launch sets in flight keep reading the previous layout
    uint32_t first = 0;
    const auto t0 = std::chrono::steady_clock::now();
    if (rc == MC_OK) rc = mc_db_add_targets(s->db, n, (const char*)dseq, (const uint64_t*)doffs, e.taxon.data(), &first);
    if (rc == MC_OK) rc = mc_db_finalize(s->db);
    if (rc == MC_OK) {
        // add + finalize return with the database stream idle: this is the device work of the extension
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        std::lock_guard<std::mutex> lk(s->mu);
        s->ext_seconds.push_back(dt);
    }
    cudaFreeAsync(dseq, cs);
    cudaFreeAsync(doffs, cs);
    cudaGetLastError();
    if (rc == MC_OK) ++*epoch_out;
    return rc;
}

}  // namespace

void mc_server::run() {
    cudaSetDevice(device);
    uint64_t seen = 0;
    for (;;) {
        std::vector<int> fin;
        std::vector<double> fin_t;
        std::vector<Extension> ext;
        std::vector<Job*> to_admit;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait(lk, [&] { return events != seen; });
            seen = events;
            if (stop && idle_locked()) return;
            fin.swap(completed);
            fin_t.swap(completed_t);
            working = true;
        }
        // 1. finished launch sets: outputs are on the host; jobs whose last
        // piece this was are done and give their device memory back
        std::vector<Job*> finished;
        for (size_t i = 0; i < fin.size(); ++i) {
            Slot& sl = slots[fin[i]];
            for (const Piece& pc : sl.pieces)
                if (--pc.job->pieces_left == 0 && pc.job->next_q >= pc.job->j.n_queries) finished.push_back(pc.job);
            sl.pieces.clear();
            for (Job* j : finished)
                if (j->t_done == 0) j->t_done = fin_t[i];
        }
        uint64_t freed = 0;
        for (Job* j : finished) {
            if (j->dbuf) cudaFreeAsync(j->dbuf, copy_stream);
            if (j->copied) cudaEventDestroy(j->copied);
            j->dbuf = nullptr;
            j->copied = nullptr;
            freed += j->bytes;
        }
        if (!fin.empty()) {
            std::lock_guard<std::mutex> lk(mu);
            for (int sidx : fin) slots[sidx].busy = false;
            in_flight -= fin.size();
            hbm_in_use -= freed;
            for (Job* j : finished) {
                j->done = true;
                ++jobs_done;
                queries_done += j->j.n_queries;
                latencies.push_back(j->t_done - j->t_submit);
                t_last = std::max(t_last, j->t_done);
            }
        }
        if (!fin.empty()) done_cv.notify_all();

        // 2. extensions, between launch sets.  A job is classified against
        // one epoch: while a split job still has pieces to launch, the
        // extensions wait (and no new job starts, see 4).
        {
            std::lock_guard<std::mutex> lk(mu);
            const bool partial = !admitted.empty() && admitted.front()->next_q > 0;
            while (!partial && !extensions.empty()) {
                ext.push_back(std::move(extensions.front()));
                extensions.pop_front();
            }
        }
        for (Extension& e : ext) {
            uint64_t ep = 0;
            const int rc = apply_extension(this, e, &ep);
            std::lock_guard<std::mutex> lk(mu);
            ++ext_applied;
            if (rc == MC_OK) {
                epoch += ep;
                ++n_ext;
            }
        }
        if (!ext.empty()) done_cv.notify_all();

        // 3. admission by device memory, in arrival order
        {
            std::lock_guard<std::mutex> lk(mu);
            while (!arrivals.empty() && hbm_in_use + arrivals.front()->bytes <= hbm_limit) {
                Job* j = arrivals.front();
                arrivals.pop_front();
                hbm_in_use += j->bytes;
                hbm_peak = std::max(hbm_peak, hbm_in_use);
                to_admit.push_back(j);
            }
        }
        std::vector<Job*> failed;
        for (Job* j : to_admit) {
            void* p = nullptr;
            cudaError_t e = cudaMallocAsync(&p, j->bytes, copy_stream);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->copied, cudaEventDisableTiming);
            if (e == cudaSuccess) {
                j->dbuf = (unsigned char*)p;
                const mc_job& q = j->j;
                const uint64_t sb = q.n_seq ? q.offs[q.n_seq] : 0;
                if (sb) e = cudaMemcpyAsync(j->dbuf, q.seq, sb, cudaMemcpyHostToDevice, copy_stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(j->dbuf + j->o_offs, q.offs, ((size_t)q.n_seq + 1) * 8, cudaMemcpyHostToDevice,
                                        copy_stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(j->dbuf + j->o_qoffs, q.qoffs, ((size_t)q.n_queries + 1) * 4,
                                        cudaMemcpyHostToDevice, copy_stream);
                if (e == cudaSuccess) e = cudaEventRecord(j->copied, copy_stream);
            }
            if (e != cudaSuccess) {
                cudaGetLastError();
                j->status = MC_ERR_CUDA;
                if (j->dbuf) cudaFreeAsync(j->dbuf, copy_stream);
                j->dbuf = nullptr;
                failed.push_back(j);
            }
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            for (Job* j : to_admit)
                if (j->status == MC_OK) admitted.push_back(j);
            for (Job* j : failed) {
                j->done = true;
                j->t_done = now();
                hbm_in_use -= j->bytes;
                ++jobs_done;
            }
        }
        if (!failed.empty()) done_cv.notify_all();

        // 4. launch sets on free slots (continuous batching)
        for (size_t si = 0; si < slots.size(); ++si) {
            Slot& sl = slots[si];
            std::vector<Piece> pieces;
            uint64_t ep = 0;
            {
                std::lock_guard<std::mutex> lk(mu);
                // with an extension pending only started jobs continue
                const bool ext_pending = !extensions.empty();
                auto may_start = [&](const Job* j) {
                    return j->ext_seq <= ext_applied && (j->next_q > 0 || !ext_pending);
                };
                if (sl.busy || admitted.empty() || !may_start(admitted.front())) continue;
                uint64_t nq = 0;
                while (!admitted.empty() && pieces.size() < max_set_jobs && nq < max_set_queries) {
                    Job* j = admitted.front();
                    if (!may_start(j)) break;
                    const uint32_t take =
                        (uint32_t)std::min<uint64_t>(j->j.n_queries - j->next_q, max_set_queries - nq);
                    pieces.push_back(Piece{j, j->next_q, j->next_q + take});
                    j->next_q += take;
                    ++j->pieces;
                    ++j->pieces_left;
                    nq += take;
                    if (j->next_q >= j->j.n_queries) admitted.pop_front();
                }
                sl.busy = true;
                ++in_flight;
                ++launch_sets;
                ep = epoch;
            }
            const double tl = now();
            std::vector<mc_batch> descs;
            std::vector<Job*> waited;
            for (const Piece& pc : pieces) {
                Job* j = pc.job;
                if (std::find(waited.begin(), waited.end(), j) == waited.end()) {
                    cudaStreamWaitEvent(sl.stream, j->copied, 0);
                    waited.push_back(j);
                }
                mc_batch b;
                b.n_seq = j->j.n_seq;
                b.n_queries = pc.q1 - pc.q0;
                b.seq = (const char*)j->dbuf;
                b.offs = (const uint64_t*)(j->dbuf + j->o_offs);
                b.qoffs = (const uint32_t*)(j->dbuf + j->o_qoffs) + pc.q0;
                b.label = (uint32_t*)(j->dbuf + j->o_label) + pc.q0;
                b.hits = (uint32_t*)(j->dbuf + j->o_hits) + pc.q0;
                b.top_target = (uint32_t*)(j->dbuf + j->o_top) + pc.q0;
                descs.push_back(b);
            }
            int rc = mc_plan_run(sl.plan, (uint32_t)descs.size(), descs.data(), sl.stream);
            for (const Piece& pc : pieces) {
                const mc_job& q = pc.job->j;
                const size_t n = (size_t)(pc.q1 - pc.q0) * 4;
                const size_t off = (size_t)pc.q0 * 4;
                if (!n) continue;
                cudaMemcpyAsync((char*)q.label + off, pc.job->dbuf + pc.job->o_label + off, n, cudaMemcpyDeviceToHost,
                                sl.stream);
                cudaMemcpyAsync((char*)q.hits + off, pc.job->dbuf + pc.job->o_hits + off, n, cudaMemcpyDeviceToHost,
                                sl.stream);
                if (q.top_target)
                    cudaMemcpyAsync((char*)q.top_target + off, pc.job->dbuf + pc.job->o_top + off, n,
                                    cudaMemcpyDeviceToHost, sl.stream);
            }
            {
                std::lock_guard<std::mutex> lk(mu);
                for (const Piece& pc : pieces) {
                    if (pc.job->t_launch < 0) {
                        pc.job->t_launch = tl;
                        pc.job->epoch = ep;
                    }
                    if (rc != MC_OK) pc.job->status = rc;
                }
                sl.pieces = pieces;
            }
            if (cudaLaunchHostFunc(sl.stream, on_set_done, &sl.ctx) != cudaSuccess) {
                // the set cannot report itself: wait for it here
                cudaGetLastError();
                cudaStreamSynchronize(sl.stream);
                on_set_done(&sl.ctx);
            }
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            working = false;
        }
        done_cv.notify_all();
    }
}

extern "C" {

int mc_server_create(mc_db* db, const mc_classify_params* params, const mc_server_config* config, mc_server** out) {
    if (!db || !params || !out) return mc::report_error(MC_ERR_ARG, "mc_server_create: NULL argument");
    *out = nullptr;
    mc_db_stats_t st;
    int rc = mc_db_stats(db, &st);
    if (rc) return rc;
    if (!st.finalized) return mc::report_error(MC_ERR_STATE, "mc_server_create: finalize the database first");
    auto s = std::make_unique<mc_server>();
    s->db = db;
    s->params = *params;
    const uint32_t n_streams = config && config->n_streams ? config->n_streams : 2;
    s->max_set_queries = config && config->max_set_queries ? config->max_set_queries : (1u << 21);
    s->max_set_jobs = config && config->max_set_jobs ? config->max_set_jobs : 256;
    if (n_streams > 16 || s->max_set_queries >= 0xFFFFFFF0u)
        return mc::report_error(MC_ERR_ARG, "mc_server_create: n_streams <= 16, max_set_queries < 2^32 - 16");
    cudaGetDevice(&s->device);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return MC_ERR_CUDA;
    }
    s->hbm_limit = config && config->hbm_limit ? config->hbm_limit : fr / 2;
    s->t0 = Clock::now();
    s->epoch = 0;
    if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess) return MC_ERR_CUDA;
    s->slots.resize(n_streams);
    for (uint32_t i = 0; i < n_streams; ++i) {
        Slot& sl = s->slots[i];
        sl.ctx = CallbackCtx{s.get(), (int)i};
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
            mc_server_free(s.release());
            return MC_ERR_CUDA;
        }
        if ((rc = mc_plan_create(db, params, nullptr, s->max_set_jobs, s->max_set_queries, &sl.plan))) {
            mc_server_free(s.release());
            return rc;
        }
    }
    s->th = std::thread([p = s.get()] { p->run(); });
    *out = s.release();
    return MC_OK;
}

int mc_server_submit(mc_server* s, const mc_job* job, uint64_t* job_id) {
    if (!s || !job || !job_id) return mc::report_error(MC_ERR_ARG, "mc_server_submit: NULL argument");
    if (!job->offs || (job->n_queries && (!job->seq || !job->qoffs || !job->label || !job->hits)))
        return mc::report_error(MC_ERR_ARG, "mc_server_submit: NULL input or output pointer");
    // the kernels index offs with qoffs: check both on the host
    for (uint32_t i = 0; i < job->n_seq; ++i)
        if (job->offs[i + 1] < job->offs[i])
            return mc::report_error(MC_ERR_ARG, "mc_server_submit: offsets decrease at sequence %u", i);
    if (job->n_queries) {
        for (uint32_t q = 0; q < job->n_queries; ++q)
            if (job->qoffs[q + 1] < job->qoffs[q])
                return mc::report_error(MC_ERR_ARG, "mc_server_submit: query offsets decrease at query %u", q);
        if (job->qoffs[job->n_queries] > job->n_seq)
            return mc::report_error(MC_ERR_ARG, "mc_server_submit: query offsets point past the last sequence");
    }
    auto j = std::make_unique<Job>();
    j->j = *job;
    j->bytes = job_bytes(*job, &j->o_offs, &j->o_qoffs, &j->o_label, &j->o_hits, &j->o_top);
    if (j->bytes > s->hbm_limit)
        return mc::report_error(MC_ERR_OOM, "mc_server_submit: the job needs %zu device bytes, the limit is %llu",
                                j->bytes, (unsigned long long)s->hbm_limit);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return MC_ERR_STATE;
        j->id = s->next_id++;
        j->ext_seq = s->ext_requested;
        j->t_submit = s->now();
        if (s->t_first < 0) s->t_first = j->t_submit;
        *job_id = j->id;
        ++s->jobs_submitted;
        Job* raw = j.get();
        s->jobs.emplace(j->id, std::move(j));
        if (raw->j.n_queries == 0) {
            raw->done = true;
            raw->t_done = raw->t_submit;
            ++s->jobs_done;
        } else {
            s->arrivals.push_back(raw);
        }
        ++s->events;
    }
    s->cv.notify_one();
    s->done_cv.notify_all();
    return MC_OK;
}

int mc_server_extend(mc_server* s, uint32_t n_targets, const char* seq, const uint64_t* offs, const uint32_t* taxon,
                     uint32_t* first_target_id) {
    if (!s || !offs || (n_targets && !taxon)) return mc::report_error(MC_ERR_ARG, "mc_server_extend: NULL argument");
    Extension e;
    const uint64_t nb = offs[n_targets];
    if (nb && !seq) return mc::report_error(MC_ERR_ARG, "mc_server_extend: NULL sequence");
    e.seq.assign(seq, seq + nb);
    e.offs.assign(offs, offs + n_targets + 1);
    e.taxon.assign(taxon, taxon + n_targets);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return MC_ERR_STATE;
        if (s->next_target == 0) {
            mc_db_stats_t st;
            if (mc_db_stats(s->db, &st) == MC_OK) s->next_target = (uint32_t)st.n_targets;
        }
        if (first_target_id) *first_target_id = s->next_target;
        s->next_target += n_targets;
        ++s->ext_requested;
        s->extensions.push_back(std::move(e));
        ++s->events;
    }
    s->cv.notify_one();
    return MC_OK;
}

int mc_server_wait(mc_server* s, uint64_t job_id, double timeout_s, mc_job_info* info) {
    if (!s) return MC_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return mc::report_error(MC_ERR_ARG, "mc_server_wait: unknown job id");
    Job* j = it->second.get();
    auto ready = [&] { return j->done; };
    if (timeout_s < 0) {
        s->done_cv.wait(lk, ready);
    } else if (!s->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
        return MC_ERR_TIMEOUT;
    }
    if (info) *info = mc_job_info{j->t_submit, j->t_launch, j->t_done, j->epoch, j->pieces, j->status};
    s->jobs.erase(it);
    return MC_OK;
}

int mc_server_drain(mc_server* s, double timeout_s) {
    if (!s) return MC_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto idle = [&] { return s->idle_locked(); };
    if (timeout_s < 0) {
        s->done_cv.wait(lk, idle);
    } else if (!s->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), idle)) {
        return MC_ERR_TIMEOUT;
    }
    return MC_OK;
}

int mc_server_stats_get(mc_server* s, mc_server_stats* out) {
    if (!s || !out) return MC_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof *out);
    out->jobs_submitted = s->jobs_submitted;
    out->jobs_done = s->jobs_done;
    out->queries_done = s->queries_done;
    out->launch_sets = s->launch_sets;
    out->extensions = s->n_ext;
    out->epoch = s->epoch;
    out->hbm_in_use = s->hbm_in_use;
    out->hbm_limit = s->hbm_limit;
    out->hbm_peak = s->hbm_peak;
    if (!s->latencies.empty()) {
        std::vector<double> l = s->latencies;
        std::sort(l.begin(), l.end());
        auto q = [&](double f) { return l[std::min(l.size() - 1, (size_t)(f * (double)(l.size() - 1) + 0.5))]; };
        out->p50_latency_s = q(0.50);
        out->p99_latency_s = q(0.99);
        out->max_latency_s = l.back();
    }
    out->busy_s = s->t_first < 0 ? 0 : std::max(0.0, s->t_last - s->t_first);
    for (double x : s->ext_seconds) {
        out->extension_mean_s += x / (double)s->ext_seconds.size();
        out->extension_max_s = std::max(out->extension_max_s, x);
    }
    return MC_OK;
}

void mc_server_free(mc_server* s) {
    if (!s) return;
    if (s->th.joinable()) {
        mc_server_drain(s, -1);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
            ++s->events;
        }
        s->cv.notify_one();
        s->th.join();
    }
    for (Slot& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.plan) mc_plan_free(sl.plan);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    for (auto& kv : s->jobs) {
        Job* j = kv.second.get();
        if (j->dbuf) cudaFreeAsync(j->dbuf, s->copy_stream);
        if (j->copied) cudaEventDestroy(j->copied);
    }
    if (s->copy_stream) {
        cudaStreamSynchronize(s->copy_stream);
        cudaStreamDestroy(s->copy_stream);
    }
    cudaGetLastError();
    delete s;
}

}  // extern "C"
