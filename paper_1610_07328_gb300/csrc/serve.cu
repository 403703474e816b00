// serve.cu -- a serving loop over a set of indexes with continuous batching.
//
// Clients submit queries (host samples) and inserts from any thread. One
// worker thread owns the indexes and the GPU work: it keeps several batch
// plans ("slots", each its own stream, buffers and CUDA graph; as many as the
// free device memory admits at creation), and whenever a slot is free and
// queries are waiting it packs up to max_batch of them into the slot, copies
// them to the device and launches the slot's batch without waiting, so the
// batches of several slots overlap on the GPU while new arrivals queue up.
// Completed slots hand their rows back to the requests. Candidate buffers are
// admitted by free device memory: a batch whose candidates outgrow its slot's
// pair buffers grows them only while reserve_bytes of device memory stay free;
// otherwise its queries go back to the front of the queue and later batches
// are admitted at half the size (doubling again after each batch that fits),
// and a single query that still does not fit is answered SSH_EBUSY. Inserts are applied
// between batches: the worker stops admitting queries, lets the slots drain,
// appends the waiting series to the indexes (Algorithm 1) and resumes; the
// plans then rewrite their table descriptors in place. A request's latency is
// measured from its arrival time (the submit time, or a scheduled arrival the
// client passes, on the server's clock) to the moment its rows are ready.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ssh_internal.cuh"

namespace ssh {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t ticket;
    int32_t length;
    double t_arrival;
    std::vector<float> x;
};

struct Result {
    ssh_status status = SSH_OK;
    std::vector<int64_t> ids;
    std::vector<float> dists;
    int32_t which = -1;
    double latency_ms = 0.0;
};

struct Insert {
    std::vector<float> x;
    std::vector<int32_t> lengths;
    double t_arrival;
};

struct Slot {
    ssh_batch* b = nullptr;
    float* d_q = nullptr;       // [max_batch * max_len] device
    float* h_q = nullptr;       // the same, pinned host staging
    int64_t* h_ids = nullptr;   // [max_batch][k] pinned
    float* h_dists = nullptr;   // [max_batch][k] pinned
    int32_t* h_which = nullptr; // [max_batch] pinned
    std::vector<Request> reqs;  // the batch in flight
    std::vector<int32_t> lengths;
    bool running = false;
};

}  // namespace
}  // namespace ssh

using namespace ssh;

struct ssh_server {
    std::vector<ssh_index*> handles;
    std::vector<int32_t> known_lengths;
    int k = 0, max_batch = 0, max_len = 0;
    int batch_cap = 0;          // queries admitted per batch now (max_batch, halved by refused growth)
    int64_t reserve_bytes = 0;  // device memory kept free when pair buffers grow
    std::vector<Slot> slots;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> pending;
    std::deque<Insert> inserts;
    std::unordered_map<int64_t, Result> done;
    std::deque<int64_t> done_order;
    int64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    ssh_server_stats st{};
    std::vector<double> batch_sizes;
    std::string worker_error;
    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace ssh {
namespace {

bool length_known(const ssh_server* s, int32_t m) {
    return std::find(s->known_lengths.begin(), s->known_lengths.end(), m) != s->known_lengths.end();
}

// Deliver a finished slot's rows to its requests (called by the worker, lock not held).
void complete_slot(ssh_server* s, Slot& sl) {
    ssh_status status = batch_finish(sl.b, s->reserve_bytes);
    const int64_t n = (int64_t)sl.reqs.size();
    if (status == SSH_EBUSY && n > 1) {
        // memory admission refused the growth: requeue the batch in order, admit smaller ones
        std::lock_guard<std::mutex> lock(s->mu);
        for (int64_t i = n - 1; i >= 0; --i) s->pending.push_front(std::move(sl.reqs[i]));
        s->batch_cap = std::max<int>(1, (int)(n / 2));
        s->st.deferred += n;
        sl.reqs.clear();
        sl.running = false;
        return;
    }
    if (status == SSH_OK) s->batch_cap = std::min(s->max_batch, 2 * s->batch_cap);
    if (status == SSH_OK) {
        const int64_t* d_ids;
        const float* d_dists;
        const int32_t* d_which;
        batch_outputs(sl.b, &d_ids, &d_dists, &d_which);
        cudaStream_t st = batch_stream(sl.b);
        cudaError_t e = cudaMemcpyAsync(sl.h_ids, d_ids, (size_t)n * s->k * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_dists, d_dists, (size_t)n * s->k * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_which, d_which, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) status = cuda_status(e, "server results");
    }
    const double t_done = s->now();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        for (int64_t i = 0; i < n; ++i) {
            Result r;
            r.status = status;
            if (status == SSH_OK) {
                r.ids.assign(sl.h_ids + i * s->k, sl.h_ids + (i + 1) * s->k);
                r.dists.assign(sl.h_dists + i * s->k, sl.h_dists + (i + 1) * s->k);
                r.which = sl.h_which[i];
            }
            r.latency_ms = (t_done - sl.reqs[i].t_arrival) * 1e3;
            s->done[sl.reqs[i].ticket] = std::move(r);
            s->done_order.push_back(sl.reqs[i].ticket);
        }
        s->st.queries_done += n;
        s->st.batches += 1;
        if (status == SSH_EBUSY) {
            s->st.refused += n;  // one query whose candidates do not fit the admitted memory
            s->worker_error = ssh_last_error();
        } else if (status != SSH_OK) {
            s->st.errors += n;
            s->worker_error = ssh_last_error();
        }
    }
    sl.reqs.clear();
    sl.running = false;
    s->cv_done.notify_all();
}

// Append the waiting series to the indexes (no slot is running).
void apply_inserts(ssh_server* s, std::deque<Insert>& batch) {
    for (Insert& ins : batch) {
        // group the series by the handle that serves their length (the first storing it)
        int64_t off = 0, i = 0;
        const int64_t n = (int64_t)ins.lengths.size();
        while (i < n) {
            const int32_t m = ins.lengths[i];
            int64_t j = i;
            int64_t len_sum = 0;
            while (j < n && ins.lengths[j] == m) len_sum += ins.lengths[j++];
            ssh_index* target = s->handles[0];
            for (ssh_index* h : s->handles)
                if (h->subs.count(m) && h->subs.at(m).count > 0) {
                    target = h;
                    break;
                }
            int64_t first = 0;
            const ssh_status st = ssh_index_add(target, ins.x.data() + off, ins.lengths.data() + i, j - i, &first);
            std::lock_guard<std::mutex> lock(s->mu);
            if (st == SSH_OK) {
                s->st.inserts_applied += j - i;
            } else {
                s->st.insert_errors += j - i;
                s->worker_error = ssh_last_error();
            }
            off += len_sum;
            i = j;
        }
        std::lock_guard<std::mutex> lock(s->mu);
        s->st.insert_latency_ms_sum += (s->now() - ins.t_arrival) * 1e3;
        s->st.insert_batches += 1;
    }
}

void worker_loop(ssh_server* s) {
    cudaSetDevice(s->handles[0]->device);
    while (true) {
        // 1. finished slots hand their rows back
        for (Slot& sl : s->slots)
            if (sl.running && batch_done(sl.b)) complete_slot(s, sl);
        int running = 0;
        for (Slot& sl : s->slots) running += sl.running;
        std::unique_lock<std::mutex> lock(s->mu);
        if (s->stop && s->pending.empty() && s->inserts.empty() && running == 0) break;
        // 2. inserts wait for the slots to drain, then go in before more queries
        if (!s->inserts.empty()) {
            if (running == 0) {
                std::deque<Insert> batch;
                batch.swap(s->inserts);
                lock.unlock();
                apply_inserts(s, batch);
                continue;
            }
        } else {
            // 3. admit waiting queries into free slots
            for (Slot& sl : s->slots) {
                if (sl.running || s->pending.empty()) continue;
                const int64_t n = std::min<int64_t>((int64_t)s->pending.size(), s->batch_cap);
                sl.reqs.clear();
                sl.lengths.clear();
                int64_t off = 0;
                for (int64_t i = 0; i < n; ++i) {
                    Request r = std::move(s->pending.front());
                    s->pending.pop_front();
                    memcpy(sl.h_q + off, r.x.data(), r.x.size() * sizeof(float));
                    off += (int64_t)r.x.size();
                    sl.lengths.push_back(r.length);
                    sl.reqs.push_back(std::move(r));
                }
                s->batch_sizes.push_back((double)n);
                lock.unlock();
                ssh_status status = SSH_OK;
                cudaError_t e = cudaMemcpyAsync(sl.d_q, sl.h_q, (size_t)off * sizeof(float), cudaMemcpyHostToDevice,
                                                batch_stream(sl.b));
                if (e != cudaSuccess) status = cuda_status(e, "server query copy");
                if (status == SSH_OK) status = batch_prepare(sl.b, sl.d_q, sl.lengths.data(), n);
                int on_device = 0;  // batches of other slots still executing on the GPU
                for (Slot& o : s->slots)
                    if (&o != &sl && o.running && !batch_done(o.b)) ++on_device;
                if (status == SSH_OK) status = batch_launch(sl.b);
                sl.running = true;
                if (status != SSH_OK) {
                    // reported through the requests: finish is skipped, rows stay empty
                    cudaStreamSynchronize(batch_stream(sl.b));
                    std::lock_guard<std::mutex> lk(s->mu);
                    for (Request& r : sl.reqs) {
                        Result res;
                        res.status = status;
                        res.latency_ms = (s->now() - r.t_arrival) * 1e3;
                        s->done[r.ticket] = std::move(res);
                        s->done_order.push_back(r.ticket);
                    }
                    s->st.errors += (int64_t)sl.reqs.size();
                    s->worker_error = ssh_last_error();
                    sl.reqs.clear();
                    sl.running = false;
                    s->cv_done.notify_all();
                }
                lock.lock();
                int r2 = 0;
                for (Slot& q : s->slots) r2 += q.running;
                s->st.max_inflight = std::max<int64_t>(s->st.max_inflight, r2);
                if (sl.running)
                    s->st.max_inflight_device = std::max<int64_t>(s->st.max_inflight_device, on_device + 1);
            }
        }
        // 4. idle: wait briefly for arrivals or completions
        running = 0;
        for (Slot& sl : s->slots) running += sl.running;
        if (running > 0) {
            lock.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        } else if (s->pending.empty() && s->inserts.empty() && !s->stop) {
            s->cv_work.wait_for(lock, std::chrono::milliseconds(2));
        }
    }
}

}  // namespace
}  // namespace ssh

extern "C" {

ssh_status ssh_server_create(ssh_index* const* handles, int nh, int k, int max_batch, int max_slots,
                             int64_t reserve_bytes, ssh_server** out) {
    return ssh_server_create_ex(handles, nh, k, max_batch, max_slots, reserve_bytes, 0, out);
}

ssh_status ssh_server_create_ex(ssh_index* const* handles, int nh, int k, int max_batch, int max_slots,
                                int64_t reserve_bytes, int64_t max_pairs, ssh_server** out) {
    if (!out) return fail_status(SSH_EINVAL, "out is NULL");
    if (reserve_bytes < 0 || max_pairs < 0) return fail_status(SSH_EINVAL, "reserve_bytes and max_pairs must be >= 0");
    *out = nullptr;
    if (!handles || nh < 1) return fail_status(SSH_EINVAL, "no indexes");
    if (max_batch < 1 || max_batch > 65535) return fail_status(SSH_EINVAL, "max_batch outside [1, 65535]");
    if (max_slots < 1 || max_slots > 64) return fail_status(SSH_EINVAL, "max_slots outside [1, 64]");
    if (k < 1 || k > kMaxTopK) return fail_status(SSH_EINVAL, "k = %d outside [1, %d]", k, kMaxTopK);
    for (int h = 0; h < nh; ++h)
        if (!handles[h] || handles[h]->family != 0)
            return fail_status(handles[h] ? SSH_ENOTSUP : SSH_EINVAL, "index %d is NULL or SRP (served indexes hash with SSH)", h);
    SSH_TRY(check_device(handles[0]));
    ssh_server* s = new ssh_server();
    s->handles.assign(handles, handles + nh);
    s->k = k;
    s->max_batch = max_batch;
    s->batch_cap = max_batch;
    s->reserve_bytes = reserve_bytes;
    s->t0 = Clock::now();
    for (ssh_index* h : s->handles)
        for (auto& kv : h->subs)
            if (kv.second.count > 0 && !length_known(s, kv.first)) {
                s->known_lengths.push_back(kv.first);
                s->max_len = std::max(s->max_len, kv.first);
            }
    ssh_status status = SSH_OK;
    // slots while the device keeps reserve_bytes free (at least one)
    for (int i = 0; i < max_slots && status == SSH_OK; ++i) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) break;
        if (i > 0 && s->slots.size() > 0 &&
            (int64_t)free_b - (int64_t)batch_device_bytes(s->slots[0].b) < reserve_bytes)
            break;
        Slot sl;
        status = ssh_batch_create(handles, nh, max_batch, k, max_pairs, &sl.b);
        if (status != SSH_OK) {
            if (i > 0) status = SSH_OK;  // keep the slots made so far
            break;
        }
        // slots overlap on the GPU: the per-class rerank shares the SMs, while the persistent
        // rerank (a cooperative launch over every SM) would wait for the other slots to drain
        ssh_batch_set_persistent(sl.b, 0);
        const size_t qbytes = (size_t)max_batch * std::max(s->max_len, 1) * sizeof(float);
        cudaError_t e = cudaMalloc(&sl.d_q, qbytes);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_q, qbytes);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_ids, (size_t)max_batch * k * 8);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_dists, (size_t)max_batch * k * 4);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_which, (size_t)max_batch * 4);
        s->slots.push_back(sl);
        if (e != cudaSuccess) status = cuda_status(e, "server slot buffers");
    }
    if (status != SSH_OK || s->slots.empty()) {
        if (status == SSH_OK) status = fail_status(SSH_ENOMEM, "no slot fits in device memory");
        ssh_server_destroy(s);
        return status;
    }
    s->st.slots = (int64_t)s->slots.size();
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return SSH_OK;
}

double ssh_server_now(const ssh_server* s) { return s ? s->now() : 0.0; }

ssh_status ssh_server_submit(ssh_server* s, const float* queries, const int32_t* lengths, int64_t n,
                             const double* arrival_s, int64_t* tickets) {
    if (!s || n < 0 || (n > 0 && (!queries || !lengths || !tickets))) return fail_status(SSH_EINVAL, "bad arguments");
    for (int64_t i = 0; i < n; ++i)
        if (!length_known(s, lengths[i]))
            return fail_status(SSH_ELENGTH, "query %lld has length %d, which no index of the server stores",
                               (long long)i, lengths[i]);
    const double t = s->now();
    std::vector<Request> rs(n);
    int64_t off = 0;
    for (int64_t i = 0; i < n; ++i) {
        rs[i].length = lengths[i];
        rs[i].t_arrival = arrival_s ? arrival_s[i] : t;
        rs[i].x.assign(queries + off, queries + off + lengths[i]);
        off += lengths[i];
    }
    {
        std::lock_guard<std::mutex> lock(s->mu);
        for (int64_t i = 0; i < n; ++i) {
            rs[i].ticket = s->next_ticket++;
            tickets[i] = rs[i].ticket;
            s->pending.push_back(std::move(rs[i]));
        }
        s->st.queries_submitted += n;
    }
    s->cv_work.notify_one();
    return SSH_OK;
}

ssh_status ssh_server_insert(ssh_server* s, const float* series, const int32_t* lengths, int64_t count) {
    if (!s || count < 0 || (count > 0 && (!series || !lengths))) return fail_status(SSH_EINVAL, "bad arguments");
    Insert ins;
    ins.t_arrival = s->now();
    int64_t total = 0;
    for (int64_t i = 0; i < count; ++i) {
        if (lengths[i] <= 0) return fail_status(SSH_ELENGTH, "series %lld has length %d", (long long)i, lengths[i]);
        total += lengths[i];
    }
    ins.x.assign(series, series + total);
    ins.lengths.assign(lengths, lengths + count);
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->inserts.push_back(std::move(ins));
        s->st.inserts_submitted += count;
    }
    s->cv_work.notify_one();
    return SSH_OK;
}

ssh_status ssh_server_wait(ssh_server* s, int64_t ticket, double timeout_s, int64_t* ids, float* dists,
                           int32_t* which, double* latency_ms) {
    if (!s || !ids || !dists) return fail_status(SSH_EINVAL, "bad arguments");
    std::unique_lock<std::mutex> lock(s->mu);
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    while (!s->done.count(ticket)) {
        if (s->cv_done.wait_until(lock, deadline) == std::cv_status::timeout && !s->done.count(ticket))
            return fail_status(SSH_ETIMEOUT, "ticket %lld not done within %.3f s", (long long)ticket, timeout_s);
    }
    Result r = std::move(s->done[ticket]);
    s->done.erase(ticket);
    s->done_order.erase(std::find(s->done_order.begin(), s->done_order.end(), ticket));
    lock.unlock();
    if (r.status != SSH_OK) return fail_status(r.status, "request %lld failed: %s", (long long)ticket, s->worker_error.c_str());
    memcpy(ids, r.ids.data(), s->k * sizeof(int64_t));
    memcpy(dists, r.dists.data(), s->k * sizeof(float));
    if (which) *which = r.which;
    if (latency_ms) *latency_ms = r.latency_ms;
    return SSH_OK;
}

ssh_status ssh_server_collect(ssh_server* s, int64_t max_n, double timeout_s, int64_t* tickets, int64_t* ids,
                              float* dists, double* latency_ms, int32_t* status, int64_t* n_out) {
    if (!s || !tickets || !n_out || max_n < 0) return fail_status(SSH_EINVAL, "bad arguments");
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->done_order.empty() && timeout_s > 0)
        s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), [&] { return !s->done_order.empty(); });
    int64_t n = 0;
    while (n < max_n && !s->done_order.empty()) {
        const int64_t t = s->done_order.front();
        s->done_order.pop_front();
        Result& r = s->done[t];
        tickets[n] = t;
        if (ids && r.status == SSH_OK) memcpy(ids + n * s->k, r.ids.data(), s->k * sizeof(int64_t));
        if (dists && r.status == SSH_OK) memcpy(dists + n * s->k, r.dists.data(), s->k * sizeof(float));
        if (latency_ms) latency_ms[n] = r.latency_ms;
        if (status) status[n] = (int32_t)r.status;
        s->done.erase(t);
        ++n;
    }
    *n_out = n;
    return SSH_OK;
}

ssh_status ssh_server_flush(ssh_server* s, double timeout_s) {
    if (!s) return fail_status(SSH_EINVAL, "NULL server");
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    while (true) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            const bool idle = s->pending.empty() && s->inserts.empty() &&
                              s->st.queries_done + s->st.errors >= s->st.queries_submitted &&
                              s->st.inserts_applied + s->st.insert_errors >= s->st.inserts_submitted;
            if (idle) return SSH_OK;
        }
        if (Clock::now() > deadline) return fail_status(SSH_ETIMEOUT, "server not idle within %.3f s", timeout_s);
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

ssh_status ssh_server_get_stats(ssh_server* s, ssh_server_stats* out) {
    if (!s || !out) return fail_status(SSH_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->st;
    double sum = 0.0;
    for (double v : s->batch_sizes) sum += v;
    out->mean_batch = s->batch_sizes.empty() ? 0.0 : sum / (double)s->batch_sizes.size();
    return SSH_OK;
}

void ssh_server_destroy(ssh_server* s) {
    if (!s) return;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        s->worker.join();
    }
    cudaSetDevice(s->handles[0]->device);
    for (Slot& sl : s->slots) {
        if (sl.b) ssh_batch_destroy(sl.b);
        cudaFree(sl.d_q);
        cudaFreeHost(sl.h_q);
        cudaFreeHost(sl.h_ids);
        cudaFreeHost(sl.h_dists);
        cudaFreeHost(sl.h_which);
    }
    delete s;
}

}  // extern "C"
