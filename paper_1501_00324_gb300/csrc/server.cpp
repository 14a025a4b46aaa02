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
//
// With grouping on (srv_set_grouping), requests on the same matrix are solved
// together as the columns of a lockstep multi-RHS CG (one group per matrix, a
// fixed width per matrix): one pass over the matrix serves every column.  A
// request takes the group when at least two of its matrix wait or the group
// already holds two (a lone right-hand side is faster on the single path).  It
// joins a free column at the group's next outer step and leaves at the outer
// step that finishes it, so columns are refilled while the group runs; its x is
// bitwise the same as cg_solve_multi of that right-hand side alone with the
// group's width.  Requests the groups cannot take (BF16, the single-reduction
// flag, options other than the group's) take the single path.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cg_run.h"
#include "multi_group.h"

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
    bool in_slot = false;       // running on the single path (not in a group)
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
    MultiGroup* group = nullptr;  // lockstep group of this matrix (grouping on)
    int64_t group_bytes = 0;
};

}  // namespace
}  // namespace fespmv

struct fespmv_server {
    int device = 0;
    int64_t budget = 0;
    int64_t used = 0;           // workspace bytes held (busy + idle)
    int max_active = 0;
    int group_width = 0;        // 0: no groups; -1: per matrix by size; else the width
    bool admit_dirty = true;    // something changed since admission last found nothing to start
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
    int64_t submitted = 0, completed = 0, peak_active = 0, peak_bytes = 0, grouped = 0;
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
        for (MatrixEntry& m : S->mats) {
            const bool spare = !m.idle.empty() || (m.group && group_empty(m.group));
            if (spare && (!victim || m.last_used < victim->last_used)) victim = &m;
        }
        if (!victim) return false;
        if (!victim->idle.empty()) {
            CgWork* w = victim->idle.back();
            victim->idle.pop_back();
            S->used -= w->bytes;
            destroy_work(w);
        } else {
            group_destroy(victim->group);
            victim->group = nullptr;
            S->used -= victim->group_bytes;
            victim->group_bytes = 0;
        }
    }
    return true;
}

static int active_groups(const fespmv_server* S) {
    int k = 0;
    for (const MatrixEntry& m : S->mats) k += m.group && !group_empty(m.group);
    return k;
}

static void finish_request(fespmv_server* S, Request* q, int rc) {
    q->rc = rc;
    if (rc != FESPMV_OK) q->error = fespmv_last_error();
    q->state = RQ_DONE;
    q->t_done = now_s();
    S->cv_done.notify_all();
}

// Requests a group can take: FP64 or FP32 refinement, no flags but reliable
// updates and NO_PRECOND.
static bool groupable(const fespmv_server* S, const MatrixEntry& m, const Request* q) {
    if (S->group_width == 0 || m.A->format != FESPMV_FMT_SLICED || m.A->max_lanes_log2 != 0 || m.A->n == 0)
        return false;
    if (q->o.precision != FESPMV_CG_F64 && q->o.precision != FESPMV_CG_F32_REFINE) return false;
    if (q->o.flags & ~(FESPMV_CG_RELIABLE | FESPMV_CG_NO_PRECOND | FESPMV_IO_HOST)) return false;
    return !m.group || group_empty(m.group) || group_matches(m.group, q->o);
}

// Try to put queue entry `q` into its matrix's group.  Returns 1 when admitted
// (or failed for good), 0 when it must wait.  Lock held.
static int admit_to_group(fespmv_server* S, Request* q) {
    MatrixEntry& m = S->mats[(size_t)q->matrix];
    if (m.group && group_empty(m.group) && !group_matches(m.group, q->o)) {
        group_destroy(m.group);   // an idle group with other options: rebuild it
        m.group = nullptr;
        S->used -= m.group_bytes;
        m.group_bytes = 0;
    }
    if (!m.group) {
        if ((int)S->active.size() + active_groups(S) >= S->max_active) return 0;
        const int kw = S->group_width > 0 ? S->group_width : group_width_auto(m.A);
        const int64_t need = group_bytes(m.A, kw);
        if (need > S->budget) {   // never fits: take the single path instead
            return -1;
        }
        if (!make_room(S, need)) return 0;
        MultiGroup* g = nullptr;
        int rc = group_create(m.A, kw, q->o, &g);
        if (rc) {
            finish_request(S, q, rc);
            return 1;
        }
        m.group = g;
        m.group_bytes = group_device_bytes(g);
        S->used += m.group_bytes;
        if (S->used > S->peak_bytes) S->peak_bytes = S->used;
    }
    if (group_empty(m.group) && (int)S->active.size() + active_groups(S) >= S->max_active) return 0;
    if (group_free_columns(m.group) == 0) return 0;
    int rc = group_add(m.group, q->ticket, q->b.data(), q->o);
    if (rc) {
        finish_request(S, q, rc);
        return 1;
    }
    m.last_used = now_s();
    q->state = RQ_RUNNING;
    q->t_start = now_s();
    q->b.clear();
    q->b.shrink_to_fit();
    const int64_t act = (int64_t)S->active.size() + active_groups(S);
    if (act > S->peak_active) S->peak_active = act;
    return 1;
}

// Admit what can start now.  Requests for groups are taken wherever they stand in
// the queue (a full group does not hold up the others); the single path starts
// the first of its requests in arrival order.  Lock held.
static bool admit_single(fespmv_server* S, std::deque<Request*>::iterator pos);

// Columns of m's group in use (waiting or solving).
static int group_load(const MatrixEntry& m) {
    return m.group ? (int)group_width_of(m.group) - group_free_columns(m.group) : 0;
}

static bool admit_one(fespmv_server* S) {
    // a group pays off when it holds two or more right-hand sides: requests take it
    // when at least two of their matrix wait in the queue or its group already
    // holds two; a lone request takes the single path
    std::vector<int> waiting(S->mats.size(), 0);
    if (S->group_width != 0)
        for (const Request* q : S->queue)
            if (groupable(S, S->mats[(size_t)q->matrix], q)) ++waiting[(size_t)q->matrix];
    bool single_blocked = false;
    for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
        Request* q = *it;
        const MatrixEntry& m = S->mats[(size_t)q->matrix];
        int r = -1;
        if (groupable(S, m, q) && (waiting[(size_t)q->matrix] >= 2 || group_load(m) >= 2))
            r = admit_to_group(S, q);
        if (r == 1) {
            if (q->state == RQ_RUNNING) ++S->grouped;
            S->queue.erase(it);
            return true;
        }
        if (r == 0) continue;
        if (single_blocked) continue;
        if (admit_single(S, it)) return true;
        single_blocked = true;
    }
    return false;
}

// Try to start queue entry *pos on the single path.  Lock held.
static bool admit_single(fespmv_server* S, std::deque<Request*>::iterator pos) {
    if ((int)S->active.size() + active_groups(S) >= S->max_active) return false;
    Request* q = *pos;
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
            S->queue.erase(pos);
            S->cv_done.notify_all();
            return true;
        }
        S->used += w->bytes;
        if (S->used > S->peak_bytes) S->peak_bytes = S->used;
    }
    S->queue.erase(pos);
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
    q->in_slot = true;
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
    const int64_t act = (int64_t)S->active.size() + active_groups(S);
    if (act > S->peak_active) S->peak_active = act;
    return true;
}

static void scheduler(fespmv_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lock(S->mu);
    for (;;) {
        // a scan of a long queue that finds nothing is repeated only after a
        // submission, a finished solve or column, or freed memory
        if (S->admit_dirty) {
            S->admit_dirty = false;
            while (admit_one(S)) {
            }
        }
        const bool groups_busy = active_groups(S) > 0;
        if (S->stop && S->active.empty() && S->queue.empty() && !groups_busy) break;
        if (S->active.empty() && !groups_busy) {
            S->cv_work.wait(lock);
            continue;
        }
        // advance every active solve without holding the lock (groups are touched by
        // this thread only)
        std::vector<Slot> work;
        work.swap(S->active);
        std::vector<MatrixEntry*> groups;
        for (MatrixEntry& m : S->mats)
            if (m.group && !group_empty(m.group)) groups.push_back(&m);
        lock.unlock();
        bool any = false;
        std::vector<GroupDone> gdone;
        std::vector<std::pair<MatrixEntry*, int>> gfail;
        for (MatrixEntry* m : groups) {
            bool progress = false;
            int rc = group_step(m->group, &progress, gdone);
            if (rc) gfail.emplace_back(m, rc);
            any |= progress;
        }
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
        for (GroupDone& d : gdone) {
            auto t = S->tickets.find(d.tag);
            if (t == S->tickets.end()) continue;
            Request* q = t->second;
            q->res = d.res;
            q->x = std::move(d.x);
            q->rc = d.res.status;
            if (q->rc != FESPMV_OK) q->error = "the solve did not converge";
            q->t_done = now_s();
            q->state = RQ_DONE;
            ++S->completed;
        }
        for (auto& f : gfail) {   // a CUDA error in a group: its requests fail, the group goes
            const std::string err = fespmv_last_error();
            for (auto& kv : S->tickets) {
                Request* q = kv.second;
                if (q->state == RQ_RUNNING && q->matrix == (int)(f.first - S->mats.data()) && !q->in_slot) {
                    q->rc = f.second;
                    q->error = err;
                    q->state = RQ_DONE;
                    q->t_done = now_s();
                }
            }
            group_destroy(f.first->group);
            f.first->group = nullptr;
            S->used -= f.first->group_bytes;
            f.first->group_bytes = 0;
        }
        if (!gdone.empty() || !gfail.empty()) {
            S->cv_done.notify_all();
            S->admit_dirty = true;
        }
        for (Slot& sl : done) {
            sl.req->state = RQ_DONE;
            ++S->completed;
            release_work(S, S->mats[(size_t)sl.req->matrix], sl.w);
            S->free_streams.push_back(sl.s);
        }
        for (Slot& sl : still) S->active.push_back(sl);
        if (!done.empty()) {
            S->cv_done.notify_all();
            S->admit_dirty = true;
        }
        if (!any && done.empty() && gdone.empty()) {
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

int srv_set_grouping(fespmv_server_t S, int32_t width) {
    if (!S || !(width == 0 || width == -1 || width == 4 || width == 8 || width == 16 || width == 32)) {
        set_error("srv_set_grouping: width must be 0, -1, 4, 8, 16 or 32");
        return FESPMV_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(S->mu);
    S->group_width = width;
    S->admit_dirty = true;
    return FESPMV_OK;
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
        S->admit_dirty = true;
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
    st->active = (int64_t)S->active.size() + active_groups(S);
    st->peak_active = S->peak_active;
    st->workspace_bytes = S->used;
    st->peak_workspace_bytes = S->peak_bytes;
    st->grouped = S->grouped;
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
    for (MatrixEntry& m : S->mats) {
        for (CgWork* w : m.idle) destroy_work(w);
        if (m.group) group_destroy(m.group);
    }
    for (cudaStream_t s : S->free_streams) cudaStreamDestroy(s);
    for (auto& kv : S->tickets) delete kv.second;
    delete S;
}

}  // extern "C"
