// Continuous-batching solve server (host runtime around the solve kernels).
//
// Requests (operator id, right-hand sides in host memory) are queued per
// operator.  A scheduler thread repeatedly
//   1. retires finished batches (event query on each slot's stream), copies the
//      solutions out of the slot's pinned buffer into each request's result and
//      records its latency (submit -> completion);
//   2. for every operator with queued requests and no batch in flight, takes
//      requests in arrival order until max_batch_rhs right-hand sides, makes the
//      operator resident (building it on the GPU on first use, after evicting
//      idle least-recently-used operators until the HBM budget admits it), and
//      launches one multi-RHS solve on a free slot: H2D copy, the power-series
//      solve, D2H copy, event record, all on the slot's stream.
// Batches of different operators run on different streams and overlap on the
// device; requests that arrive while others run join the next batch of their
// operator as soon as its previous batch retires.  One handle never has two
// batches in flight (its workspace is per handle).  When the resident operators
// exceed the HBM budget (every operator was busy at admission), idle operators
// with no queued requests are evicted, least recently used first, as soon as
// batches retire.
#include "hm_internal.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

using namespace hm;

namespace {

using clk = std::chrono::steady_clock;

struct Request {
    int64_t id;
    int op;
    int nrhs;
    std::vector<float2> b;    // N x nrhs, column-major
    std::vector<float2> x;
    clk::time_point t_submit, t_done;
    bool done = false;
    hm_status status = HM_OK;
};

struct Operator {
    int basis = HM_RWG;
    std::vector<double> xyz;
    std::vector<int32_t> cells;
    std::vector<double> eps_r;
    double wavelength;
    hm_build_opts bo;
    hm_solve_opts so;
    hm_matrix h = nullptr;
    int64_t n = 0;
    int64_t bytes = 0;         // device bytes when resident (estimate before the first build)
    bool busy = false;
    clk::time_point last_use;
    std::deque<int64_t> queue;
    int builds = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    float2 *h_buf = nullptr;   // pinned: b then x
    float2 *d_b = nullptr, *d_x = nullptr;
    size_t cap = 0;            // complex elements per half
    bool busy = false;
    int op = -1;
    std::vector<int64_t> reqs;
    int nrhs = 0;
    // device-loop mode: 1 = posted to the ring at ring_idx, 2 = result being copied out
    int stage = 0;
    int64_t ring_idx = -1;
};

} // namespace

struct hm_server_s {
    int max_batch_rhs;
    int64_t budget;
    std::vector<Slot> slots;
    std::vector<Operator> ops;
    std::map<int64_t, Request> reqs;
    int64_t next_id = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    std::atomic<bool> stop{false};
    hm_status fatal = HM_OK;
    std::string fatal_msg;
    int device = 0;
    // statistics
    int64_t batches = 0, solved_rhs = 0, evictions = 0, builds = 0;
    int64_t resident_bytes = 0, peak_resident = 0;
    // device-resident request loop (device_loop mode): the ring and control words in
    // mapped pinned host memory (host and device addresses), the loop's device words,
    // its stream and grid; the recorded phase lists per (operator, slot, RHS bucket)
    bool device_loop = false;
    hm::LoopEntry *ring = nullptr, *d_ring = nullptr;
    hm::LoopCtl *ctl = nullptr, *d_ctl = nullptr;
    hm::LoopDev *d_dev = nullptr;
    unsigned *d_bar = nullptr;
    int *d_loop_status = nullptr;
    cudaStream_t loop_stream = nullptr;
    int loop_grid = 0;
    bool loop_running = false;
    int64_t ring_next = 0;         // next ring index to post
    int64_t loop_head = 0;         // first ring index the next loop launch serves
    std::map<std::pair<int, int>, std::pair<const hm::Phase *, int>> recorded;   // (operator, RHS bucket)
    int64_t loop_launches = 0, loop_stops = 0;
};

namespace {

void drop_operator(hm_server_s *S, int op);

hm_status slot_reserve(Slot &s, size_t elems)
{
    if (s.cap >= elems) return HM_OK;
    if (s.h_buf) cudaFreeHost(s.h_buf);
    if (s.d_b) cudaFree(s.d_b);
    if (s.d_x) cudaFree(s.d_x);
    s.h_buf = nullptr; s.d_b = s.d_x = nullptr; s.cap = 0;
    HM_CUDA(cudaMallocHost((void **)&s.h_buf, 2 * elems * sizeof(float2)));
    HM_CUDA(cudaMalloc((void **)&s.d_b, elems * sizeof(float2)));
    HM_CUDA(cudaMalloc((void **)&s.d_x, elems * sizeof(float2)));
    s.cap = elems;
    return HM_OK;
}

// make operator op resident, evicting idle LRU operators to respect the budget
hm_status make_resident(hm_server_s *S, int op)
{
    Operator &o = S->ops[op];
    if (o.h) return HM_OK;
    const int64_t need = o.bytes;
    while (S->resident_bytes + need > S->budget) {
        int victim = -1;
        for (int i = 0; i < (int)S->ops.size(); ++i) {
            const Operator &c = S->ops[i];
            if (c.h && !c.busy && (victim < 0 || c.last_use < S->ops[victim].last_use)) victim = i;
        }
        if (victim < 0) break;   // everything resident is in use: admit anyway, the budget is a target
        drop_operator(S, victim);
        S->resident_bytes -= S->ops[victim].bytes;
        S->evictions++;
    }
    const int per = o.basis == HM_SWG ? 4 : 3;
    hm_mesh mesh{o.basis, (int64_t)o.xyz.size() / 3, o.xyz.data(), (int64_t)o.cells.size() / per, o.cells.data(),
                 o.eps_r.empty() ? nullptr : o.eps_r.data(), o.wavelength};
    hm_matrix h = nullptr;
    hm_status st = hm_build(&mesh, &o.bo, nullptr, &h);
    if (st != HM_OK) return st;
    st = hm_factor_leaf(h, nullptr);
    if (st != HM_OK) {
        hm_destroy(h);
        return st;
    }
    hm_info info;
    hm_get_info(h, &info);
    o.h = h;
    o.n = info.n;
    o.bytes = info.device_bytes;
    o.builds++;
    S->builds++;
    S->resident_bytes += o.bytes;
    S->peak_resident = std::max(S->peak_resident, S->resident_bytes);
    return HM_OK;
}

void retire(hm_server_s *S, Slot &s)
{
    const int64_t N = S->ops[s.op].n;
    const float2 *hx = s.h_buf + s.cap;
    int col = 0;
    const auto now = clk::now();
    for (int64_t id : s.reqs) {
        Request &r = S->reqs[id];
        r.x.assign(hx + (size_t)col * N, hx + (size_t)(col + r.nrhs) * N);
        col += r.nrhs;
        r.t_done = now;
        r.done = true;
    }
    // the operator's footprint grows with its workspace (right-hand-side vectors)
    hm_info info;
    if (hm_get_info(S->ops[s.op].h, &info) == HM_OK) {
        S->resident_bytes += info.device_bytes - S->ops[s.op].bytes;
        S->ops[s.op].bytes = info.device_bytes;
        S->peak_resident = std::max(S->peak_resident, S->resident_bytes);
    }
    S->ops[s.op].busy = false;
    S->ops[s.op].last_use = now;
    S->solved_rhs += s.nrhs;
    s.busy = false;
    s.reqs.clear();
    s.op = -1;
}

void fail_requests(hm_server_s *S, int op, hm_status st)
{
    Operator &o = S->ops[op];
    for (int64_t id : o.queue) {
        Request &r = S->reqs[id];
        r.status = st;
        r.done = true;
        r.t_done = clk::now();
    }
    o.queue.clear();
}

// ---- device-resident request loop ----------------------------------------------------
//
// One cooperative kernel (k_serve_loop) stays on the GPU and serves batches from a
// ring in mapped pinned host memory: the scheduler copies a batch's right-hand
// sides into its slot's device buffer, writes the ring entry (the batch's recorded
// one-launch phase list and its operator's context) and marks it ready; the loop
// runs it without any launch and marks it done; the scheduler then copies the
// solutions out on the slot's stream.  Work that needs the GPU otherwise (builds,
// allocation, recording a new phase list) is done while the loop is stopped: a
// stop entry after everything posted makes it leave once those are served.  An
// idle loop leaves by itself after LOOP_IDLE_POLLS polls (about a second) and is
// launched again when the next batch is posted.

constexpr int RING = 64;
constexpr uint32_t LOOP_IDLE_POLLS = 400000;
constexpr int RHS_BUCKET = 4;        // batches are padded to a multiple of 4 right-hand sides

int ring_state(hm_server_s *S, int64_t idx) { return __atomic_load_n(&S->ring[idx % RING].state, __ATOMIC_ACQUIRE); }
void ring_set(hm_server_s *S, int64_t idx, int v) { __atomic_store_n(&S->ring[idx % RING].state, v, __ATOMIC_RELEASE); }

// collects a loop kernel that has left (its stream), and where it stopped
void loop_reap(hm_server_s *S)
{
    if (!S->loop_running || __atomic_load_n(&S->ctl->exited, __ATOMIC_ACQUIRE) == 0) return;
    cudaStreamSynchronize(S->loop_stream);
    S->loop_running = false;
    S->loop_head = __atomic_load_n(&S->ctl->head, __ATOMIC_ACQUIRE);
}

hm_status loop_start(hm_server_s *S)
{
    __atomic_store_n(&S->ctl->start, S->loop_head, __ATOMIC_RELAXED);
    __atomic_store_n(&S->ctl->head, S->loop_head, __ATOMIC_RELAXED);
    __atomic_store_n(&S->ctl->exited, 0, __ATOMIC_RELEASE);
    HM_CUDA(cudaMemsetAsync(S->d_loop_status, 0, sizeof(int), S->loop_stream));
    hm_status st = launch_serve_loop(S->d_ring, RING, S->d_ctl, S->d_dev, S->d_bar, S->d_loop_status, S->loop_grid,
                                     LOOP_IDLE_POLLS, S->loop_stream);
    if (st != HM_OK) return st;
    S->loop_running = true;
    S->loop_launches++;
    return HM_OK;
}

// stops the loop (after everything posted is served) so that the host may use the GPU
hm_status loop_stop(hm_server_s *S, std::unique_lock<std::mutex> &lk)
{
    loop_reap(S);
    if (!S->loop_running) return HM_OK;
    const int64_t idx = S->ring_next;
    ring_set(S, idx, LOOP_STOP);
    const auto deadline = clk::now() + std::chrono::seconds(60);
    while (__atomic_load_n(&S->ctl->exited, __ATOMIC_ACQUIRE) == 0) {
        if (clk::now() > deadline) return fail(HM_ERR_TIMEOUT, "the serving loop did not stop within 60 s");
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
    }
    loop_reap(S);
    ring_set(S, idx, LOOP_FREE);
    S->loop_stops++;
    return HM_OK;
}

// destroys an operator's handle; its recorded phase lists go with it
void drop_operator(hm_server_s *S, int op)
{
    hm_destroy(S->ops[op].h);
    S->ops[op].h = nullptr;
    for (auto it = S->recorded.begin(); it != S->recorded.end();)
        it = it->first.first == op ? S->recorded.erase(it) : std::next(it);
}

int bucket_of(int nrhs, int max_rhs)
{
    const int b = (nrhs + RHS_BUCKET - 1) / RHS_BUCKET * RHS_BUCKET;
    return std::min(b, (max_rhs + RHS_BUCKET - 1) / RHS_BUCKET * RHS_BUCKET);
}

void fail_slot(hm_server_s *S, Slot &slot, hm_status st)
{
    for (int64_t id : slot.reqs) {
        Request &r = S->reqs[id];
        r.status = st;
        r.done = true;
        r.t_done = clk::now();
    }
    S->ops[slot.op].busy = false;
    slot.busy = false;
    slot.stage = 0;
    slot.reqs.clear();
    slot.op = -1;
    S->cv_done.notify_all();
}

// the scheduler of the device-loop mode
void loop_device(hm_server_s *S)
{
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        bool progressed = false;
        // 1. batches the loop has served: copy their solutions out; retire copied ones
        for (Slot &s : S->slots) {
            if (!s.busy) continue;
            if (s.stage == 1 && ring_state(S, s.ring_idx) == LOOP_DONE) {
                const int64_t N = S->ops[s.op].n;
                cudaMemcpyAsync(s.h_buf + s.cap, s.d_x, sizeof(float2) * N * s.nrhs, cudaMemcpyDeviceToHost, s.stream);
                cudaEventRecord(s.done, s.stream);
                ring_set(S, s.ring_idx, LOOP_FREE);
                s.stage = 2;
                progressed = true;
            }
            if (s.stage == 2) {
                const cudaError_t e = cudaEventQuery(s.done);
                if (e == cudaSuccess) {
                    retire(S, s);
                    s.stage = 0;
                    progressed = true;
                } else if (e != cudaErrorNotReady) {
                    S->fatal = HM_ERR_CUDA;
                    S->fatal_msg = cudaGetErrorString(e);
                    S->stop = true;
                }
            }
        }
        if (progressed) S->cv_done.notify_all();
        // over the budget with nothing posted: stop the loop and evict idle operators without
        // queued requests, least recently used first (freeing memory must not wait on the loop)
        if (S->resident_bytes > S->budget) {
            bool idle = true;
            for (Slot &q : S->slots) idle &= !q.busy;
            auto victim_of = [&] {
                int v = -1;
                for (int i = 0; i < (int)S->ops.size(); ++i) {
                    const Operator &c = S->ops[i];
                    if (c.h && !c.busy && c.queue.empty() && (v < 0 || c.last_use < S->ops[v].last_use)) v = i;
                }
                return v;
            };
            if (idle && victim_of() >= 0 && loop_stop(S, lk) == HM_OK) {
                int v;
                while (S->resident_bytes > S->budget && (v = victim_of()) >= 0) {
                    drop_operator(S, v);
                    S->resident_bytes -= S->ops[v].bytes;
                    S->evictions++;
                }
            }
        }
        // 2. a loop that left on an error (a bounded wait gave up) leaves its current batch unserved
        loop_reap(S);
        if (!S->loop_running) {
            int lst = 0;
            cudaMemcpy(&lst, S->d_loop_status, sizeof(int), cudaMemcpyDeviceToHost);
            if (lst != 0) {
                for (Slot &s : S->slots)
                    if (s.busy && s.stage == 1 && s.ring_idx == S->loop_head) {
                        ring_set(S, s.ring_idx, LOOP_FREE);
                        fail_slot(S, s, (hm_status)lst);
                    }
                S->loop_head++;
                cudaMemset(S->d_loop_status, 0, sizeof(int));
            }
            // a loop that left on idle just before a batch was posted: launch it again
            bool pending = false;
            for (Slot &s : S->slots) pending |= s.busy && s.stage == 1;
            if (pending && loop_start(S) != HM_OK) {
                S->fatal = HM_ERR_CUDA;
                S->fatal_msg = "the serving loop could not be launched";
                S->stop = true;
            }
        }
        // 3. post new batches
        for (int op = 0; op < (int)S->ops.size(); ++op) {
            Operator &o = S->ops[op];
            if (o.busy || o.queue.empty()) continue;
            int si = -1;
            for (int q = 0; q < (int)S->slots.size(); ++q)
                if (!S->slots[q].busy) { si = q; break; }
            if (si < 0) break;
            Slot &slot = S->slots[si];
            std::vector<int64_t> take;
            int nrhs = 0;
            while (!o.queue.empty()) {
                const Request &r = S->reqs[o.queue.front()];
                if (!take.empty() && nrhs + r.nrhs > S->max_batch_rhs) break;
                take.push_back(o.queue.front());
                nrhs += r.nrhs;
                o.queue.pop_front();
            }
            const int bucket = bucket_of(nrhs, S->max_batch_rhs);
            const int top = bucket_of(S->max_batch_rhs, S->max_batch_rhs);
            hm_status st = HM_OK;
            const auto key = std::make_pair(op, bucket);
            if (!o.h || !S->recorded.count(key) || slot.cap < (size_t)o.n * top) {
                // host-side GPU work: stop the loop first (everything posted is served before it leaves)
                if ((st = loop_stop(S, lk)) == HM_OK && (st = make_resident(S, op)) == HM_OK)
                    st = slot_reserve(slot, (size_t)o.n * top);   // this slot is free
                // every bucket of the operator at once, the largest first, so that the handle's
                // workspace never grows later (a regrowth would free the lists already recorded);
                // the lists do not depend on the slot (its buffers are passed with each batch)
                for (int b = top; st == HM_OK && b >= RHS_BUCKET; b -= RHS_BUCKET) {
                    const auto k2 = std::make_pair(op, b);
                    if (S->recorded.count(k2)) continue;
                    const Phase *ph = nullptr;
                    int n = 0;
                    if ((st = persist_phases(o.h, slot.d_b, slot.d_x, b, &o.so, &ph, &n)) == HM_OK)
                        S->recorded[k2] = {ph, n};
                }
                if (st == HM_OK) {
                    hm_info info;
                    if (hm_get_info(o.h, &info) == HM_OK) {
                        S->resident_bytes += info.device_bytes - o.bytes;
                        o.bytes = info.device_bytes;
                        S->peak_resident = std::max(S->peak_resident, S->resident_bytes);
                    }
                }
            }
            if (st != HM_OK) {
                for (int64_t id : take) { S->reqs[id].status = st; S->reqs[id].done = true; }
                S->cv_done.notify_all();
                continue;
            }
            const int64_t N = o.n;
            int col = 0;
            for (int64_t id : take) {
                const Request &r = S->reqs[id];
                std::memcpy(slot.h_buf + (size_t)col * N, r.b.data(), sizeof(float2) * N * r.nrhs);
                col += r.nrhs;
            }
            std::memset(slot.h_buf + (size_t)nrhs * N, 0, sizeof(float2) * N * (bucket - nrhs));
            cudaMemcpyAsync(slot.d_b, slot.h_buf, sizeof(float2) * N * bucket, cudaMemcpyHostToDevice, slot.stream);
            if (cudaStreamSynchronize(slot.stream) != cudaSuccess) {
                for (int64_t id : take) { S->reqs[id].status = HM_ERR_CUDA; S->reqs[id].done = true; }
                S->cv_done.notify_all();
                continue;
            }
            const auto &rec = S->recorded[key];
            const int64_t idx = S->ring_next++;
            LoopEntry &e = S->ring[idx % RING];
            e.n_phases = rec.second;
            e.phases = rec.first;
            e.b = slot.d_b;
            e.x = slot.d_x;
            persist_ctx(o.h, &e.ctx);
            ring_set(S, idx, LOOP_READY);
            slot.busy = true;
            slot.stage = 1;
            slot.ring_idx = idx;
            slot.op = op;
            slot.reqs = take;
            slot.nrhs = nrhs;
            o.busy = true;
            o.last_use = clk::now();
            S->batches++;
            progressed = true;
            loop_reap(S);
            if (!S->loop_running && (st = loop_start(S)) != HM_OK) {
                S->fatal = st;
                S->fatal_msg = "the serving loop could not be launched";
                S->stop = true;
            }
        }
        if (!progressed) {
            bool any_busy = false;
            for (Slot &s : S->slots) any_busy |= s.busy;
            if (any_busy) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(5));
                lk.lock();
            } else {
                S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
            }
        }
    }
    loop_stop(S, lk);
}

void loop(hm_server_s *S)
{
    cudaSetDevice(S->device);
    if (S->device_loop) {
        loop_device(S);
        return;
    }
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        bool progressed = false;
        // 1. retire finished batches
        for (Slot &s : S->slots) {
            if (!s.busy) continue;
            const cudaError_t e = cudaEventQuery(s.done);
            if (e == cudaSuccess) {
                retire(S, s);
                progressed = true;
            } else if (e != cudaErrorNotReady) {
                S->fatal = HM_ERR_CUDA;
                S->fatal_msg = cudaGetErrorString(e);
                S->stop = true;
            }
        }
        if (progressed) {
            S->cv_done.notify_all();
            // shrink to the budget: evict idle operators without queued requests, LRU first
            while (S->resident_bytes > S->budget) {
                int victim = -1;
                for (int i = 0; i < (int)S->ops.size(); ++i) {
                    const Operator &c = S->ops[i];
                    if (c.h && !c.busy && c.queue.empty() &&
                        (victim < 0 || c.last_use < S->ops[victim].last_use))
                        victim = i;
                }
                if (victim < 0) break;
                hm_destroy(S->ops[victim].h);
                S->ops[victim].h = nullptr;
                S->resident_bytes -= S->ops[victim].bytes;
                S->evictions++;
            }
        }
        // 2. launch new batches
        for (int op = 0; op < (int)S->ops.size(); ++op) {
            Operator &o = S->ops[op];
            if (o.busy || o.queue.empty()) continue;
            Slot *slot = nullptr;
            for (Slot &s : S->slots)
                if (!s.busy) { slot = &s; break; }
            if (!slot) break;
            hm_status st = make_resident(S, op);
            if (st != HM_OK) {
                fail_requests(S, op, st);
                S->cv_done.notify_all();
                continue;
            }
            // take requests in arrival order up to max_batch_rhs right-hand sides
            std::vector<int64_t> take;
            int nrhs = 0;
            while (!o.queue.empty()) {
                const Request &r = S->reqs[o.queue.front()];
                if (!take.empty() && nrhs + r.nrhs > S->max_batch_rhs) break;
                take.push_back(o.queue.front());
                nrhs += r.nrhs;
                o.queue.pop_front();
            }
            const int64_t N = o.n;
            st = slot_reserve(*slot, (size_t)N * nrhs);
            if (st != HM_OK) {
                for (int64_t id : take) { S->reqs[id].status = st; S->reqs[id].done = true; }
                S->cv_done.notify_all();
                continue;
            }
            int col = 0;
            for (int64_t id : take) {
                const Request &r = S->reqs[id];
                std::memcpy(slot->h_buf + (size_t)col * N, r.b.data(), sizeof(float2) * N * r.nrhs);
                col += r.nrhs;
            }
            cudaMemcpyAsync(slot->d_b, slot->h_buf, sizeof(float2) * N * nrhs, cudaMemcpyHostToDevice, slot->stream);
            st = hm_powerseries_solve(o.h, slot->d_b, N, slot->d_x, N, nrhs, &o.so, slot->stream, nullptr);
            if (st != HM_OK) {
                for (int64_t id : take) { S->reqs[id].status = st; S->reqs[id].done = true; }
                S->cv_done.notify_all();
                continue;
            }
            cudaMemcpyAsync(slot->h_buf + slot->cap, slot->d_x, sizeof(float2) * N * nrhs, cudaMemcpyDeviceToHost,
                            slot->stream);
            cudaEventRecord(slot->done, slot->stream);
            slot->busy = true;
            slot->op = op;
            slot->reqs = take;
            slot->nrhs = nrhs;
            o.busy = true;
            o.last_use = clk::now();
            S->batches++;
            progressed = true;
        }
        if (!progressed) {
            bool any_busy = false;
            for (Slot &s : S->slots) any_busy |= s.busy;
            if (any_busy) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            } else {
                S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
            }
        }
    }
}

} // namespace

using namespace hm;

extern "C" {

hm_status hm_server_create_ex(int n_slots, int64_t hbm_budget_bytes, int max_batch_rhs, int device_loop,
                              hm_server *out)
{
    if (!out || n_slots < 1 || n_slots > 32 || hbm_budget_bytes <= 0 || max_batch_rhs < 1)
        return fail(HM_ERR_ARG, "bad server arguments");
    *out = nullptr;
    hm_server S = new hm_server_s();
    S->max_batch_rhs = max_batch_rhs;
    S->budget = hbm_budget_bytes;
    S->device_loop = device_loop != 0;
    cudaGetDevice(&S->device);
    S->slots.resize(n_slots);
    for (Slot &s : S->slots) {
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) {
            hm_server_destroy(S);
            return fail(HM_ERR_CUDA, "stream or event creation failed");
        }
    }
    if (S->device_loop) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, S->device);
        S->loop_grid = serve_loop_grid(sms);
        bool ok = cudaHostAlloc((void **)&S->ring, RING * sizeof(LoopEntry), cudaHostAllocMapped) == cudaSuccess &&
                  cudaHostAlloc((void **)&S->ctl, sizeof(LoopCtl), cudaHostAllocMapped) == cudaSuccess;
        if (ok) {
            std::memset(S->ring, 0, RING * sizeof(LoopEntry));
            std::memset(S->ctl, 0, sizeof(LoopCtl));
            ok = cudaHostGetDevicePointer((void **)&S->d_ring, S->ring, 0) == cudaSuccess &&
                 cudaHostGetDevicePointer((void **)&S->d_ctl, S->ctl, 0) == cudaSuccess &&
                 cudaMalloc((void **)&S->d_dev, sizeof(LoopDev)) == cudaSuccess &&
                 cudaMalloc((void **)&S->d_bar, 2 * sizeof(unsigned)) == cudaSuccess &&
                 cudaMalloc((void **)&S->d_loop_status, sizeof(int)) == cudaSuccess &&
                 cudaMemset(S->d_loop_status, 0, sizeof(int)) == cudaSuccess &&
                 cudaStreamCreateWithFlags(&S->loop_stream, cudaStreamNonBlocking) == cudaSuccess;
        }
        if (!ok) {
            hm_server_destroy(S);
            return fail(HM_ERR_OOM, "the serving loop's ring or device words could not be allocated");
        }
    }
    S->worker = std::thread(loop, S);
    *out = S;
    return HM_OK;
}

hm_status hm_server_create(int n_slots, int64_t hbm_budget_bytes, int max_batch_rhs, hm_server *out)
{
    return hm_server_create_ex(n_slots, hbm_budget_bytes, max_batch_rhs, 0, out);
}

hm_status hm_server_add_mesh(hm_server S, const hm_mesh *mesh, const hm_build_opts *bo, const hm_solve_opts *so,
                             int *op_id, int64_t *n_unknowns)
{
    if (!S || !mesh || !bo || !so || !op_id) return fail(HM_ERR_ARG, "bad operator arguments");
    int64_t nunk = 0;
    hm_status st = count_unknowns(mesh, &nunk);
    if (st != HM_OK) return st;
    if (mesh->basis == HM_SWG) {
        if (!mesh->eps_r) return fail(HM_ERR_ARG, "eps_r is required for an SWG mesh");
        for (int64_t t = 0; t < mesh->n_cell; ++t)
            if (!(mesh->eps_r[t] > 0) || !std::isfinite(mesh->eps_r[t]))
                return fail(HM_ERR_ARG, "eps_r must be finite and > 0");
    }
    if (so->fp64) return fail(HM_ERR_ARG, "the server runs the complex64 path");
    Operator o;
    const int per = mesh->basis == HM_SWG ? 4 : 3;
    o.basis = mesh->basis;
    o.xyz.assign(mesh->xyz, mesh->xyz + 3 * mesh->n_vert);
    o.cells.assign(mesh->cells, mesh->cells + per * mesh->n_cell);
    if (mesh->basis == HM_SWG) o.eps_r.assign(mesh->eps_r, mesh->eps_r + mesh->n_cell);
    o.wavelength = mesh->wavelength;
    o.bo = *bo;
    o.bo.keep_fp64 = 0;
    o.so = *so;
    o.n = nunk;
    // size estimate before the first build: ~60 KB per unknown
    o.bytes = nunk * 60 * 1024;
    o.last_use = clk::now();
    std::lock_guard<std::mutex> lk(S->mu);
    S->ops.push_back(std::move(o));
    *op_id = (int)S->ops.size() - 1;
    if (n_unknowns) *n_unknowns = nunk;
    return HM_OK;
}

hm_status hm_server_submit(hm_server S, int op_id, const void *b, int64_t n, int nrhs, int64_t *req_id)
{
    if (!S || !b || !req_id || nrhs < 1) return fail(HM_ERR_ARG, "bad request");
    std::unique_lock<std::mutex> lk(S->mu);
    if (op_id < 0 || op_id >= (int)S->ops.size()) return fail(HM_ERR_ARG, "unknown operator");
    if (n != S->ops[op_id].n) return fail(HM_ERR_ARG, "right-hand side length differs from the operator's N");
    if (nrhs > S->max_batch_rhs) return fail(HM_ERR_ARG, "request has more right-hand sides than max_batch_rhs");
    if (S->fatal != HM_OK) return fail(S->fatal, S->fatal_msg);
    {
        // the request's own device footprint, at least: its right-hand sides and solutions in
        // a slot's device buffers plus the leaf-level solve's 16 work vectors per column
        // (more with more levels or the residual's slots).  A request that cannot fit the
        // HBM budget even alone is refused here, before it is queued; queued requests are
        // not affected.
        const Operator &o = S->ops[op_id];
        const int m = o.so.n_levels > 0 ? o.so.n_levels : 1;
        const int64_t per_rhs = (int64_t)sizeof(float2) * n * (2 + 4 * (m + 1) + 8);
        if ((int64_t)nrhs * per_rhs > S->budget)
            return fail(HM_ERR_OOM, "request needs at least " + std::to_string((int64_t)nrhs * per_rhs) +
                                        " device bytes, above the server's HBM budget");
    }
    Request r;
    r.id = S->next_id++;
    r.op = op_id;
    r.nrhs = nrhs;
    r.b.assign((const float2 *)b, (const float2 *)b + (size_t)n * nrhs);
    r.t_submit = clk::now();
    const int64_t id = r.id;
    S->reqs.emplace(id, std::move(r));
    S->ops[op_id].queue.push_back(id);
    *req_id = id;
    lk.unlock();
    S->cv_work.notify_one();
    return HM_OK;
}

hm_status hm_server_wait(hm_server S, int64_t req_id, void *x, double *latency_ms)
{
    if (!S || !x) return fail(HM_ERR_ARG, "null argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return fail(HM_ERR_ARG, "unknown request id");
    const auto deadline = clk::now() + std::chrono::seconds(600);
    while (!it->second.done && S->fatal == HM_OK) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout)
            return fail(HM_ERR_TIMEOUT, "request did not complete within 600 s");
    }
    if (!it->second.done) return fail(S->fatal, S->fatal_msg);
    Request r = std::move(it->second);
    S->reqs.erase(it);
    if (r.status != HM_OK) return fail(r.status, "request failed");
    std::memcpy(x, r.x.data(), r.x.size() * sizeof(float2));
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
    return HM_OK;
}

hm_status hm_server_get_info(hm_server S, hm_server_info *st)
{
    if (!S || !st) return fail(HM_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    st->batches = S->batches;
    st->solved_rhs = S->solved_rhs;
    st->builds = S->builds;
    st->evictions = S->evictions;
    st->resident_bytes = S->resident_bytes;
    st->peak_resident_bytes = S->peak_resident;
    st->loop_launches = S->loop_launches;
    st->loop_stops = S->loop_stops;
    return HM_OK;
}

void hm_server_destroy(hm_server S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (Slot &s : S->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.h_buf) cudaFreeHost(s.h_buf);
        if (s.d_b) cudaFree(s.d_b);
        if (s.d_x) cudaFree(s.d_x);
    }
    for (Operator &o : S->ops)
        if (o.h) hm_destroy(o.h);
    if (S->loop_stream) {
        cudaStreamSynchronize(S->loop_stream);
        cudaStreamDestroy(S->loop_stream);
    }
    if (S->ring) cudaFreeHost(S->ring);
    if (S->ctl) cudaFreeHost(S->ctl);
    if (S->d_dev) cudaFree(S->d_dev);
    if (S->d_bar) cudaFree(S->d_bar);
    if (S->d_loop_status) cudaFree(S->d_loop_status);
    delete S;
}

} // extern "C"
