// Solve server: continuous batching of CG solves on one GPU (srv_* in fespmv.h).
//
// Requests (matrix id, right-hand side, options) are queued by srv_submit.  A
// scheduler thread admits them in arrival order as soon as a slot is free and
// the request's workspace fits in the byte budget (a workspace freed by a
// finished solve of the same matrix is reused, idle workspaces of other
// matrices are released when the budget needs room).  Every admitted solve
// runs on its own stream with its own workspace; the scheduler advances all of
// them round-robin, queueing each one's next iteration graph as soon as its
// previous status word is back, so iterations of many solves overlap on the
// device while matrices stay resident.  A solve in the mix runs exactly the
// kernels, grids and reduction order of cg_solve alone, so its result is
// bitwise the same.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cg_run.h"

namespace fespmv {

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum ReqState { RQ_QUEUED, RQ_RUNNING, RQ_DONE };

struct Request {
    int64_t ticket = 0;
    int matrix = 0;
    std::vector<double> b, x;
    cg_options o{};
    cg_result res{};
    int state = RQ_QUEUED;
    int rc = FESPMV_OK;
    std::string error;
    double t_submit = 0, t_start = 0, t_done = 0;
};

struct Slot {
    Request* req = nullptr;
    CgWork* w = nullptr;
    cudaStream_t s = nullptr;
    CgRun run;
};

struct MatrixEntry {
    fespmv_mat* A = nullptr;
    std::vector<CgWork*> idle;  // finished workspaces kept for reuse (their graphs too)
    int64_t bytes = 0;          // workspace bytes for this matrix
    double last_used = 0.0;
};

}  // namespace
}  // namespace fespmv

struct fespmv_server {
    int device = 0;
    int64_t budget = 0;
    int64_t used = 0;           // workspace bytes held (busy + idle)
    int max_active = 0;
    std::vector<fespmv::MatrixEntry> mats;
    std::deque<fespmv::Request*> queue;
    std::unordered_map<int64_t, fespmv::Request*> tickets;
    std::vector<fespmv::Slot> active;
    std::vector<cudaStream_t> free_streams;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread thread;
    bool stop = false;
    int64_t next_ticket = 1;
    // statistics
    int64_t submitted = 0, completed = 0, peak_active = 0, peak_bytes = 0;
};

namespace fespmv {

static void release_work(fespmv_server* S, MatrixEntry& m, CgWork* w) {
    m.idle.push_back(w);
    m.last_used = now_s();
}

// Free idle workspaces (least recently used matrix first) until `need` more
// bytes fit in the budget.  Called with the lock held.
static bool make_room(fespmv_server* S, int64_t need) {
    while (S->used + need > S->budget) {
        MatrixEntry* victim = nullptr;
        for (MatrixEntry& m : S->mats)
            if (!m.idle.empty() && (!victim || m.last_used < victim->last_used)) victim = &m;
        if (!victim) return false;
        CgWork* w = victim->idle.back();
        victim->idle.pop_back();
        S->used -= w->bytes;
        destroy_work(w);
    }
    return true;
}

// Try to start the request at the head of the queue.  Lock held.
static bool admit_one(fespmv_server* S) {
    if (S->queue.empty() || (int)S->active.size() >= S->max_active) return false;
    Request* q = S->queue.front();
    MatrixEntry& m = S->mats[(size_t)q->matrix];
    CgWork* w = nullptr;
    if (!m.idle.empty()) {
        w = m.idle.back();
        m.idle.pop_back();
    } else {
        if (!make_room(S, m.bytes)) return false;  // wait for running solves to finish
        int rc = create_work(m.A, true, &w);
        if (!rc && (m.A->d_val32 || m.A->d_val16)) rc = ensure_low_work(w);
        if (rc) {
            if (w) destroy_work(w);
            q->rc = rc;
            q->error = fespmv_last_error();
            q->state = RQ_DONE;
            q->t_done = now_s();
            S->queue.pop_front();
            S->cv_done.notify_all();
            return true;
        }
        S->used += w->bytes;
        if (S->used > S->peak_bytes) S->peak_bytes = S->used;
    }
    S->queue.pop_front();
    Slot slot;
    slot.req = q;
    slot.w = w;
    if (!S->free_streams.empty()) {
        slot.s = S->free_streams.back();
        S->free_streams.pop_back();
    } else {
        cudaStreamCreateWithFlags(&slot.s, cudaStreamNonBlocking);
    }
    q->state = RQ_RUNNING;
    q->t_start = now_s();
    CgRun& r = slot.run;
    r.A = m.A;
    r.w = w;
    r.s = slot.s;
    r.o = q->o;
    r.permute = m.A->format == FESPMV_FMT_SLICED;
    r.has_x0 = false;
    r.out_host = true;
    r.x_out = w->h_io;
    std::memcpy(w->h_io, q->b.data(), sizeof(double) * q->b.size());
    int rc = stage_inputs(r, w->h_io, nullptr, true);
    if (!rc) rc = run_begin(r);
    if (rc) {
        q->rc = rc;
        q->error = fespmv_last_error();
        r.phase = PH_DONE;
    }
    S->active.push_back(slot);
    if ((int64_t)S->active.size() > S->peak_active) S->peak_active = (int64_t)S->active.size();
    return true;
}

static void scheduler(fespmv_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lock(S->mu);
    for (;;) {
        while (admit_one(S)) {
        }
        if (S->stop && S->active.empty() && S->queue.empty()) break;
        if (S->active.empty()) {
            S->cv_work.wait(lock);
            continue;
        }
        // advance every active solve without holding the lock
        std::vector<Slot> work;
        work.swap(S->active);
        lock.unlock();
        bool any = false;
        std::vector<Slot> still, done;
        for (Slot& sl : work) {
            bool progress = false;
            if (sl.run.phase != PH_DONE && sl.req->rc == FESPMV_OK) {
                int rc = run_step(sl.run, false, &progress);
                if (rc) {
                    sl.req->rc = rc;
                    sl.req->error = fespmv_last_error();
                    sl.run.phase = PH_DONE;
                }
            }
            any |= progress;
            if (sl.run.phase == PH_DONE) {
                cudaStreamSynchronize(sl.s);
                Request* q = sl.req;
                if (q->rc == FESPMV_OK) {
                    int rc = run_result(sl.run, &q->res);
                    q->rc = rc;
                    if (rc != FESPMV_OK) q->error = fespmv_last_error();
                    if (sl.run.error == FESPMV_OK)
                        q->x.assign(sl.w->h_io, sl.w->h_io + sl.run.A->n);
                }
                q->t_done = now_s();
                done.push_back(sl);
            } else {
                still.push_back(sl);
            }
        }
        lock.lock();
        for (Slot& sl : done) {
            sl.req->state = RQ_DONE;
            ++S->completed;
            release_work(S, S->mats[(size_t)sl.req->matrix], sl.w);
            S->free_streams.push_back(sl.s);
        }
        for (Slot& sl : still) S->active.push_back(sl);
        if (!done.empty()) S->cv_done.notify_all();
        if (!any && done.empty()) {
            // nothing ready: wait briefly (new submissions wake us at once)
            S->cv_work.wait_for(lock, std::chrono::microseconds(20));
        }
    }
}

}  // namespace fespmv

using namespace fespmv;

extern "C" {

int srv_create(fespmv_server_t* out, int64_t workspace_budget_bytes, int32_t max_active) {
    if (!out || workspace_budget_bytes <= 0 || max_active <= 0) {
        set_error("srv_create: need out, a positive budget and max_active");
        return FESPMV_ERR_INVALID_ARG;
    }
    *out = nullptr;
    try {
        fespmv_server* S = new fespmv_server();
        cudaError_t e = cudaGetDevice(&S->device);
        if (e != cudaSuccess) {
            delete S;
            return cuda_fail(e, "cudaGetDevice");
        }
        S->budget = workspace_budget_bytes;
        S->max_active = max_active;
        S->thread = std::thread(scheduler, S);
        *out = S;
        return FESPMV_OK;
    } catch (...) {
        set_error("srv_create: could not start the scheduler thread");
        return FESPMV_ERR_OOM;
    }
}

int srv_register(fespmv_server_t S, fespmv_mat_t A, int32_t* matrix_id) {
    if (!S || !A || !matrix_id) {
        set_error("null argument");
        return FESPMV_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(S->mu);
    MatrixEntry m;
    m.A = A;
    m.bytes = work_bytes(A, A->d_val32 || A->d_val16);
    if (m.bytes > S->budget) {
        set_error("one solve of this matrix needs %lld workspace bytes, above the budget",
                  (long long)m.bytes);
        return FESPMV_ERR_OOM;
    }
    S->mats.push_back(m);
    *matrix_id = (int32_t)S->mats.size() - 1;
    return FESPMV_OK;
}

int srv_submit(fespmv_server_t S, int32_t matrix_id, const double* b, const cg_options* opts,
               int64_t* ticket) {
    if (!S || !ticket) {
        set_error("null argument");
        return FESPMV_ERR_INVALID_ARG;
    }
    try {
        cg_options o;
        std::memset(&o, 0, sizeof(o));
        if (opts) o = *opts;
        int rc = normalize_options(o);
        if (rc) return rc;
        if (o.flags & (FESPMV_IO_PERMUTED | FESPMV_CG_X0)) {
            set_error("srv_submit: vectors are host arrays in the input numbering, x0 = 0");
            return FESPMV_ERR_INVALID_ARG;
        }
        std::unique_lock<std::mutex> lock(S->mu);
        if (matrix_id < 0 || matrix_id >= (int32_t)S->mats.size()) {
            set_error("unknown matrix id %d", matrix_id);
            return FESPMV_ERR_INVALID_ARG;
        }
        fespmv_mat* A = S->mats[(size_t)matrix_id].A;
        if ((rc = check_precision(A, o.precision))) return rc;
        if (A->n > 0 && !b) {
            set_error("b is NULL");
            return FESPMV_ERR_INVALID_ARG;
        }
        Request* q = new Request();
        q->ticket = S->next_ticket++;
        q->matrix = matrix_id;
        q->b.assign(b, b + A->n);
        q->o = o;
        q->t_submit = now_s();
        S->tickets[q->ticket] = q;
        S->queue.push_back(q);
        ++S->submitted;
        *ticket = q->ticket;
        S->cv_work.notify_one();
        return FESPMV_OK;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return FESPMV_ERR_OOM;
    }
}

int srv_poll(fespmv_server_t S, int64_t ticket, int32_t wait, double* x, cg_result* res,
             srv_timing* timing) {
    if (!S) {
        set_error("null argument");
        return FESPMV_ERR_INVALID_ARG;
    }
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) {
        set_error("unknown ticket %lld", (long long)ticket);
        return FESPMV_ERR_INVALID_ARG;
    }
    Request* q = it->second;
    if (q->state != RQ_DONE) {
        if (!wait) return FESPMV_PENDING;
        S->cv_done.wait(lock, [&] { return q->state == RQ_DONE; });
    }
    if (x && !q->x.empty()) std::memcpy(x, q->x.data(), sizeof(double) * q->x.size());
    if (res) *res = q->res;
    if (timing) {
        timing->t_queue_s = q->t_start > 0 ? q->t_start - q->t_submit : 0.0;
        timing->t_solve_s = q->t_start > 0 ? q->t_done - q->t_start : 0.0;
        timing->t_total_s = q->t_done - q->t_submit;
    }
    const int rc = q->rc;
    if (rc != FESPMV_OK && rc != FESPMV_ERR_NOT_CONVERGED && rc != FESPMV_ERR_BREAKDOWN)
        set_error("%s", q->error.c_str());
    if (rc == FESPMV_ERR_CANCELLED && timing) timing->t_solve_s = 0.0;
    S->tickets.erase(it);
    delete q;
    return rc;
}

int srv_get_stats(fespmv_server_t S, srv_stats* st) {
    if (!S || !st) {
        set_error("null argument");
        return FESPMV_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(S->mu);
    st->submitted = S->submitted;
    st->completed = S->completed;
    st->queued = (int64_t)S->queue.size();
    st->active = (int64_t)S->active.size();
    st->peak_active = S->peak_active;
    st->workspace_bytes = S->used;
    st->peak_workspace_bytes = S->peak_bytes;
    return FESPMV_OK;
}

int srv_cancel_queued(fespmv_server_t S, int64_t* n_cancelled) {
    if (!S) {
        set_error("null argument");
        return FESPMV_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(S->mu);
    int64_t n = 0;
    const double t = now_s();
    for (Request* q : S->queue) {
        q->rc = FESPMV_ERR_CANCELLED;
        q->error = "cancelled before it started";
        q->state = RQ_DONE;
        q->t_done = t;
        ++n;
    }
    S->queue.clear();
    if (n_cancelled) *n_cancelled = n;
    S->cv_done.notify_all();
    return FESPMV_OK;
}

void srv_destroy(fespmv_server_t S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->thread.joinable()) S->thread.join();
    for (MatrixEntry& m : S->mats)
        for (CgWork* w : m.idle) destroy_work(w);
    for (cudaStream_t s : S->free_streams) cudaStreamDestroy(s);
    for (auto& kv : S->tickets) delete kv.second;
    delete S;
}

}  // extern "C"
