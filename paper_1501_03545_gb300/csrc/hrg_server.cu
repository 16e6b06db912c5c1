// hrg_server.cu -- a request loop for graph generation on one GPU.
//
// Requests (hrg_params) are queued on submit.  `slots` worker threads, each
// with its own context (whose grow-only workspace, the band structures
// included, stays resident between requests) and its own stream, take work
// whenever they are free: a worker admits the queued requests in arrival
// order while their estimated device memory fits the budget, and generates
// all of them as one batch (hrg_generate_batch_begin).  Requests that arrive
// while others run join the next batch a free worker forms, and the batches
// of different workers overlap on the device -- continuous batching.  A
// graph does not depend on what it was batched with (each graph's points and
// edges are fixed by its own parameters), so every result equals the result
// of the same request run alone.
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/hrg.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s(Clock::time_point t0) { return std::chrono::duration<double>(Clock::now() - t0).count(); }

// device memory of one batch (r, phi and row offsets in one allocation, the
// neighbour ids in another); shared by the requests it served
struct Block {
    void *head = nullptr;
    int32_t *col = nullptr;
    cudaStream_t stream = nullptr;
    int refs = 0;
    double *r = nullptr, *phi = nullptr;
    int64_t *row_off = nullptr;
};

struct Req {
    int64_t ticket = 0;
    hrg_params p{};
    size_t est_out = 0, est_work = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    int status = HRG_OK;
    bool done = false;
    std::string err;
    std::shared_ptr<Block> block;
    int64_t first_pt = 0, n_entries = 0;
    int32_t batch_size = 0;
};

}  // namespace

struct hrg_server {
    int device = 0;
    size_t budget = 0;
    int32_t max_batch = 4096;
    Clock::time_point t0 = Clock::now();
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> queue;
    std::unordered_map<int64_t, std::unique_ptr<Req>> reqs;
    int64_t next_ticket = 1;
    // in_use = outputs of unreleased requests + the workers' resident
    // workspaces (measured) + the estimated workspace growth of running batches
    size_t in_use = 0, peak_in_use = 0;
    std::vector<size_t> resident;  // per worker: its context's workspace after its last batch
    bool stop = false;
    std::vector<std::thread> workers;
    std::string err;
    // counters
    int64_t completed = 0, batches = 0, batched_requests = 0, max_running = 0, running = 0;
};

namespace {

int fail(hrg_server *s, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s) {
        std::lock_guard<std::mutex> g(s->mu);
        s->err = buf;
    }
    return code;
}

// Device bytes of a request: outputs (r, phi, row offsets, neighbour ids at
// 1.1 kbar per vertex) and the workspace of its generation (about 260 bytes
// per vertex: ~100 of band structure and per-vertex lists, 128 of kept-row
// buffer, 32 of hub-entry pool; plus the big-row sort buffer at up to 4
// bytes per entry and the pool's fixed 64 MB), with the 1/8 slack the
// workspace grows by: 300 bytes per vertex.
void estimate(const hrg_params &p, size_t &out, size_t &work)
{
    const double n = (double)p.n, e = 1.1 * p.avg_degree * n + 1024.0;
    out = (size_t)(16.0 * n + 8.0 * (n + 1) + 4.0 * e) + 4096;
    work = (size_t)(300.0 * n + 4.5 * e) + ((size_t)1 << 26);
}

void run_batch(hrg_server *s, hrg_ctx *ctx, cudaStream_t st, std::vector<Req *> &batch)
{
    const int32_t count = (int32_t)batch.size();
    std::vector<hrg_params> items(count);
    int64_t N = 0;
    for (int32_t k = 0; k < count; ++k) {
        items[k] = batch[k]->p;
        N += batch[k]->p.n;
    }
    auto blk = std::make_shared<Block>();
    blk->stream = st;
    int rc = HRG_OK;
    std::string msg;
    hrg_job *job = nullptr;
    int64_t ne = 0;
    // r, phi, row offsets first; the neighbour ids once 2m is known
    void *head = nullptr;
    const size_t head_bytes = 16 * (size_t)N + 8 * (size_t)(N + 1) + 256;
    if (cudaMallocAsync(&head, head_bytes, st) != cudaSuccess) {
        cudaGetLastError();
        rc = HRG_ENOMEM;
        msg = "device allocation for a batch failed";
    }
    if (rc == HRG_OK) {
        blk->r = (double *)head;
        blk->phi = blk->r + N;
        blk->row_off = (int64_t *)(blk->phi + N);
        rc = hrg_generate_batch_begin(ctx, count, items.data(), 0, st, blk->r, blk->phi, blk->row_off, &job, &ne);
        if (rc) msg = hrg_last_error(ctx);
    }
    void *colm = nullptr;
    if (rc == HRG_OK) {
        if (cudaMallocAsync(&colm, 4 * (size_t)(ne > 0 ? ne : 1), st) != cudaSuccess) {
            cudaGetLastError();
            rc = HRG_ENOMEM;
            msg = "device allocation for neighbour ids failed";
            hrg_job_release(job);
        }
    }
    if (rc == HRG_OK) {
        blk->col = (int32_t *)colm;
        rc = hrg_generate_finish(job, blk->col);
        if (rc) msg = hrg_last_error(ctx);
        hrg_stats stt{};
        hrg_job_stats(job, &stt);
        hrg_job_release(job);
    }
    // host copies of the row offsets at the graph boundaries
    std::vector<int64_t> firsts(count + 1, 0), pts(count + 1, 0);
    for (int32_t k = 0; k < count; ++k) pts[k + 1] = pts[k] + items[k].n;
    if (rc == HRG_OK) {
        for (int32_t k = 0; k < count; ++k) {
            if (cudaMemcpyAsync(&firsts[k], blk->row_off + pts[k], sizeof(int64_t), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess) {
                rc = HRG_ECUDA;
                msg = "read-back failed";
                break;
            }
        }
        firsts[count] = ne;
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            rc = HRG_ECUDA;
            msg = "stream synchronize failed";
        }
    }
    if (rc != HRG_OK) {
        if (colm) cudaFreeAsync(colm, st);
        if (head) cudaFreeAsync(head, st);
    } else {
        blk->head = head;
        blk->col = (int32_t *)colm;
        blk->refs = count;
    }
    const double t = now_s(s->t0);
    std::lock_guard<std::mutex> g(s->mu);
    for (int32_t k = 0; k < count; ++k) {
        Req *q = batch[k];
        q->status = rc;
        q->err = msg;
        q->t_done = t;
        q->done = true;
        q->batch_size = count;
        if (rc == HRG_OK) {
            q->block = blk;
            q->first_pt = pts[k];
            q->n_entries = firsts[k + 1] - firsts[k];
        } else {
            s->in_use -= q->est_out;
        }
        ++s->completed;
    }
    --s->running;
    ++s->batches;
    s->batched_requests += count;
    s->cv_done.notify_all();
}

void worker_main(hrg_server *s, int slot)
{
    cudaSetDevice(s->device);
    hrg_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;
    const bool ok = hrg_create(&ctx, s->device) == HRG_OK &&
                    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
    // the workspace beyond what this worker's context already holds
    const auto growth = [&](size_t work) { return work > s->resident[slot] ? work - s->resident[slot] : (size_t)0; };
    const auto fits = [&](const Req *q) { return s->in_use + q->est_out + growth(q->est_work) <= s->budget; };
    for (;;) {
        std::vector<Req *> batch;
        size_t grown = 0;  // estimated workspace growth admitted with the batch
        {
            std::unique_lock<std::mutex> g(s->mu);
            for (;;) {
                s->cv_work.wait(g, [&] {
                    return s->stop || (!s->queue.empty() && (fits(s->queue.front()) || s->resident[slot] > 0));
                });
                if (s->stop || fits(s->queue.front())) break;
                // too large while this worker idles on a resident workspace: free it
                // (the other idle workers do the same when woken)
                const size_t held = s->resident[slot];
                g.unlock();
                const bool freed = ok && hrg_release_workspace(ctx) == HRG_OK;
                g.lock();
                if (freed) {
                    s->in_use -= held;
                    s->resident[slot] = 0;
                }
                s->cv_work.notify_all();
                if (!freed) {  // cannot shrink: wait for releases
                    s->cv_work.wait(g, [&] { return s->stop || s->queue.empty() || fits(s->queue.front()); });
                    if (s->stop) break;
                }
            }
            if (s->stop) break;  // the queue was cancelled
            // admit in arrival order while the memory fits
            int64_t N = 0;
            size_t work = 0, out = 0;
            while (!s->queue.empty() && (int32_t)batch.size() < s->max_batch) {
                Req *q = s->queue.front();
                const size_t g2 = growth(work + q->est_work);
                if (s->in_use + out + q->est_out + g2 > s->budget || (!batch.empty() && N + q->p.n > 0x7fffffffLL))
                    break;
                s->queue.pop_front();
                work += q->est_work;
                out += q->est_out;
                N += q->p.n;
                q->t_start = now_s(s->t0);
                batch.push_back(q);
            }
            grown = growth(work);
            s->in_use += out + grown;
            if (s->in_use > s->peak_in_use) s->peak_in_use = s->in_use;
            if (!batch.empty()) {
                ++s->running;
                if (s->running > s->max_running) s->max_running = s->running;
            }
            // every worker: whether the next request fits depends on the worker
            // (its resident workspace), so a single wake-up could reach one that
            // cannot take it and leave the one that can asleep
            if (!s->queue.empty()) s->cv_work.notify_all();
        }
        if (batch.empty()) continue;
        if (!ok) {
            std::lock_guard<std::mutex> g(s->mu);
            for (Req *q : batch) {
                q->status = HRG_ECUDA;
                q->err = "worker could not create its context or stream";
                q->done = true;
                q->t_done = now_s(s->t0);
                s->in_use -= q->est_out;
                ++s->completed;
            }
            s->in_use -= grown;
            --s->running;
            s->cv_done.notify_all();
            continue;
        }
        run_batch(s, ctx, st, batch);
        // the estimate of the growth gives way to the workspace measured now
        int64_t held = 0;
        hrg_workspace_bytes(ctx, &held);
        std::lock_guard<std::mutex> g(s->mu);
        s->in_use = s->in_use - grown - s->resident[slot] + (size_t)held;
        s->resident[slot] = (size_t)held;
        if (s->in_use > s->peak_in_use) s->peak_in_use = s->in_use;
        s->cv_work.notify_all();
    }
    if (st) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    if (ctx) hrg_destroy(ctx);
}

}  // namespace

extern "C" int hrg_server_create(hrg_server **out, int device, int32_t slots, int64_t mem_budget_bytes)
{
    if (!out || slots < 1 || slots > 64) return HRG_EINVAL;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return HRG_ECUDA;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return HRG_ECUDA;
    auto *s = new hrg_server();
    s->device = device;
    s->budget = mem_budget_bytes > 0 ? (size_t)mem_budget_bytes : (size_t)(0.7 * (double)free_b);
    s->resident.assign(slots, 0);
    for (int k = 0; k < slots; ++k) s->workers.emplace_back(worker_main, s, k);
    *out = s;
    return HRG_OK;
}

extern "C" int hrg_server_submit(hrg_server *s, const hrg_params *p, int64_t *ticket)
{
    if (!s || !p || !ticket) return HRG_EINVAL;
    double R = 0;
    if (p->n < 2 || p->n > 0x7fffffffLL || !(p->alpha > 0.5) || p->bands < 0 || p->bands > 64)
        return fail(s, HRG_EINVAL, "invalid request parameters");
    if (!(p->R_override > 0.0) && hrg_solve_radius(p->n, p->alpha, p->avg_degree, &R) != HRG_OK)
        return fail(s, HRG_EINVAL, "no radius for n=%lld alpha=%g avg_degree=%g", (long long)p->n, p->alpha,
                    p->avg_degree);
    auto q = std::make_unique<Req>();
    q->p = *p;
    estimate(*p, q->est_out, q->est_work);
    std::lock_guard<std::mutex> g(s->mu);
    if (q->est_out + q->est_work > s->budget) {
        s->err = "request larger than the server's memory budget";
        return HRG_ENOMEM;
    }
    q->ticket = s->next_ticket++;
    q->t_submit = now_s(s->t0);
    *ticket = q->ticket;
    s->queue.push_back(q.get());
    s->reqs.emplace(q->ticket, std::move(q));
    s->cv_work.notify_all();  // all workers: only some may be able to take it
    return HRG_OK;
}

static void fill_result(const Req *q, hrg_result *out)
{
    memset(out, 0, sizeof *out);
    out->status = q->status;
    out->n = q->p.n;
    out->n_entries = q->n_entries;
    out->submit_s = q->t_submit;
    out->start_s = q->t_start;
    out->done_s = q->t_done;
    out->batch_size = q->batch_size;
    if (q->status == HRG_OK && q->block) {
        // the request's points and rows sit at its offset within the batch
        out->r = q->block->r + q->first_pt;
        out->phi = q->block->phi + q->first_pt;
        out->row_off = q->block->row_off + q->first_pt;
        out->col_idx = q->block->col;
    }
}

extern "C" int hrg_server_wait(hrg_server *s, int64_t ticket, double timeout_s, hrg_result *out)
{
    if (!s || !out) return HRG_EINVAL;
    std::unique_lock<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return HRG_EINVAL;
    Req *q = it->second.get();
    const auto pred = [&] { return q->done; };
    if (timeout_s < 0) s->cv_done.wait(g, pred);
    else if (!s->cv_done.wait_for(g, std::chrono::duration<double>(timeout_s), pred)) return HRG_ETIMEOUT;
    fill_result(q, out);
    if (q->status != HRG_OK) s->err = q->err;
    return q->status;
}

extern "C" int hrg_server_release(hrg_server *s, int64_t ticket)
{
    if (!s) return HRG_EINVAL;
    std::shared_ptr<Block> blk;
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return HRG_EINVAL;
        Req *q = it->second.get();
        if (!q->done) return HRG_ESTATE;
        if (q->status == HRG_OK) s->in_use -= q->est_out;
        blk = q->block;
        if (blk && --blk->refs == 0 && blk->head) {
            cudaSetDevice(s->device);
            cudaFreeAsync(blk->col, blk->stream);
            cudaFreeAsync(blk->head, blk->stream);
            blk->head = nullptr;
        }
        s->reqs.erase(it);
        s->cv_work.notify_all();
    }
    return HRG_OK;
}

extern "C" int hrg_server_stats(hrg_server *s, hrg_server_counters *out)
{
    if (!s || !out) return HRG_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    memset(out, 0, sizeof *out);
    out->completed = s->completed;
    out->batches = s->batches;
    out->batched_requests = s->batched_requests;
    out->queued = (int64_t)s->queue.size();
    out->max_running = s->max_running;
    out->in_use_bytes = (int64_t)s->in_use;
    out->peak_in_use_bytes = (int64_t)s->peak_in_use;
    out->budget_bytes = (int64_t)s->budget;
    size_t res = 0;
    for (size_t r : s->resident) res += r;
    out->resident_bytes = (int64_t)res;
    return HRG_OK;
}

extern "C" const char *hrg_server_last_error(hrg_server *s)
{
    if (!s) return "null server";
    std::lock_guard<std::mutex> g(s->mu);
    static thread_local std::string copy;
    copy = s->err;
    return copy.c_str();
}

extern "C" int hrg_server_destroy(hrg_server *s)
{
    if (!s) return HRG_EINVAL;
    {
        // requests still queued are cancelled; running batches finish
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        for (Req *q : s->queue) {
            q->status = HRG_ESTATE;
            q->err = "server destroyed before the request ran";
            q->done = true;
        }
        s->queue.clear();
        s->cv_work.notify_all();
        s->cv_done.notify_all();
    }
    for (auto &t : s->workers) t.join();
    // results never released
    cudaSetDevice(s->device);
    for (auto &kv : s->reqs) {
        Req *q = kv.second.get();
        if (q->block && q->block->head) {
            cudaFree(q->block->col);
            cudaFree(q->block->head);
            q->block->head = nullptr;
        }
    }
    delete s;
    return HRG_OK;
}
