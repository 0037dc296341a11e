// Serving loop of libscgal: continuous batching of MaxCut SDP solves.
//
// A worker thread owns up to max_slots resident solves.  Each round it
//   1. admits queued requests (oldest first, or -- SCGAL_ADMIT_SHORTEST_PREDICTED --
//      least predicted work first, from the iterations the finished requests of
//      the same size took) while a slot is free and the
//      request's estimated device footprint fits the remaining budget (the
//      solve's z, y, sketch and Lanczos basis then stay on the device until it
//      finishes);
//   2. enqueues the next stretch of every resident solve before waiting for
//      any of them: small FP32 instances in the batched engine's persistent
//      launches (one per kernel variant, each instance running until a time
//      budget is spent), the others as chunks of iterations on their own streams;
//   3. while those run, sets up the solves admitted in step 1 (they join the
//      next round) and retires the solves that finished in the previous round
//      (met the stopping rule of Eq. E.1 or T_max): Nystrom reconstruction,
//      rounding, result published for scgal_poll, device memory released;
//   4. waits for the round and marks the solves that finished in it.
// A request that arrives while others are mid-solve joins at the next round.
// Warm starts: a request submitted with keep_state leaves its final iterate in
// host memory; a later request on a graph of the same size that names it in
// warm_from starts from that iterate (Section 6.2's state: z, y, the sketch,
// p and tau) with the iteration counter at a quarter of its final value.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "batch.h"

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t id = 0;
    int kind = 0;                       // 0: MaxCut graph, 1: coded-diffraction phase retrieval
    std::vector<int32_t> row_ptr, col;  // MaxCut
    std::vector<double> w;
    bool has_w = false;
    std::vector<double> masks, b;       // phase retrieval: L x n masks (re, im), L n measurements
    int32_t L = 0;
    int32_t n = 0;
    int64_t nnz = 0;
    scgal_params prm{};
    double t_submit = 0, t_admit = 0;
    size_t footprint = 0;
    long long first_t = 1;              // 1, or the iteration a warm start resumed at
    double predicted_iters = 0;         // the work model's estimate when the request was queued
};

// Iterations to finish (gap and infeasibility at tol, else T_max) of the
// requests served so far, by size bucket: floor(log2 n) and the average degree
// rounded to a multiple of four.  Each bucket keeps the mean of log iterations;
// a new request is predicted from its bucket, else the nearest bucket of the
// same degree, else all buckets, else T_max / 2.
struct WorkModel {
    std::map<std::pair<int, int>, std::pair<double, long long>> b;   // (sum of log T, count)
    static std::pair<int, int> key(int n, long long nnz) {
        int lg = 0;
        while ((2LL << lg) <= n) ++lg;
        const int deg = (int)((nnz / std::max(1, n) + 2) / 4) * 4;
        return {lg, deg};
    }
    void add(int n, long long nnz, long long iters) {
        auto& e = b[key(n, nnz)];
        e.first += std::log((double)std::max<long long>(1, iters));
        ++e.second;
    }
    double predict(int n, long long nnz, int T_max) const {
        const auto k = key(n, nnz);
        auto it = b.find(k);
        if (it != b.end()) return std::exp(it->second.first / it->second.second);
        double best = -1, dist = 1e9, all = 0;
        long long cnt = 0;
        for (const auto& e : b) {
            all += e.second.first;
            cnt += e.second.second;
            if (e.first.second == k.second && std::abs(e.first.first - k.first) < dist) {
                dist = std::abs(e.first.first - k.first);
                best = std::exp(e.second.first / e.second.second);
            }
        }
        if (best > 0) return best;
        if (cnt) return std::exp(all / cnt);
        return 0.5 * T_max;
    }
};

// Final iterate of a finished request submitted with keep_state (host copies).
struct Saved {
    int n = 0, R = 0, prec = 0;
    std::vector<double> z, y, S;
    double sc[4] = {0, 0, 0, 0};        // p, tau, t, converged (scgal_get_state)
    size_t bytes() const { return sizeof(double) * (z.size() + y.size() + S.size()); }
};

struct Slot {
    scgal_t h = nullptr;
    Request req;
    bool active = false;
    bool batched = false;   // advanced by the batched kernel (else by the handle's graphs)
    int variant = 0;        // batched kernel variant
    bool fin = false;       // finished; retired during the next round
    int fin_status = 0;
    bool fin_has_st = false;
    scgal_stats fin_st{};
};

// Device bytes of one FP32 solve (mirrors the handle's allocations, with margin).
size_t estimate_footprint(int n, long long nnz, const scgal_params& p) {
    const double q = std::ceil(std::pow((double)p.T_max, 0.25) * std::log((double)n));
    const double qmax = std::min<double>(q, n - 1);
    const double ldb = (double)((n + 63) / 64 * 64);
    const double vb = p.precision == 64 ? 8.0 : 4.0;
    double bytes = 4.0 * (n + 1) + 4.0 * nnz + vb * nnz          // CSR (values only for general weights)
                   + vb * (qmax + 1) * ldb                       // Lanczos basis
                   + vb * 4.0 * n                                // Y, v, cdiag, dvec
                   + (p.omega == SCGAL_OMEGA_REGEN ? 1.0 : 2.0) * vb * n * p.R   // S, and Omega unless regenerated
                   + 16.0 * n                                    // z, y
                   + 2.0 * 16.0 * n * p.R                        // reconstruction Y, U (FP64)
                   + 60.0 * p.T_max + 8.0 * 65 * 1216 + 65536    // history, q table, partials, scalars
                   + 8.0 * nnz + 24.0 * n;                       // sliced layout of the batched engine
    return (size_t)(bytes * 1.15);
}

// Device bytes of one phase-retrieval solve (complex vectors; mirrors the
// handle's allocations, with margin).
size_t estimate_footprint_phase(int n, int L, const scgal_params& p) {
    const double q = std::ceil(std::pow((double)p.T_max, 0.25) * std::log((double)n));
    const double qmax = std::min<double>(q, n - 1);
    const double ldb = (double)((n + 63) / 64 * 64);
    const double vb = p.precision == 64 ? 16.0 : 8.0;   // complex element
    const double d = (double)L * n;
    double bytes = vb * (qmax + 1) * ldb                          // Lanczos basis
                   + vb * (L + 2) * ldb                           // D x planes, v
                   + (p.omega == SCGAL_OMEGA_REGEN ? 1.0 : 2.0) * vb * n * p.R   // S, and Omega unless regenerated
                   + vb * (2.0 * d + n)                           // masks, FFT scratch, twiddles
                   + 0.5 * vb * d + 24.0 * d                      // weights; z, y, b
                   + 2.0 * 16.0 * n * p.R                         // reconstruction Y, U (complex FP64)
                   + 60.0 * p.T_max + 8.0 * 65 * 4096 + 65536;    // history, q table, partials, scalars
    return (size_t)(bytes * 1.15);
}

}  // namespace

struct scgal_server {
    size_t budget = 0;
    int max_slots = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    std::map<uint64_t, scgal_result> done;
    std::vector<Slot> slots;
    std::thread worker;
    bool stopping = false;
    uint64_t next_id = 1;
    size_t in_use = 0, peak = 0;
    long long submitted = 0, admitted = 0, completed = 0, rejected = 0;
    double wait_ms = 0, admit_ms = 0, retire_ms = 0;   // worker time per phase (guarded by mu)
    long long rounds_done = 0;
    int active = 0;
    static constexpr int CHUNK = 8;          // iterations per graph-path slot per round
    static constexpr unsigned long long BATCH_BUDGET_NS = 25000000ull;   // batched launch time per round
    static constexpr size_t QUEUE_MAX = 1 << 16;
    // iterates kept for warm starts (keep_state requests), oldest dropped past the cap
    std::map<uint64_t, Saved> saved;
    std::deque<uint64_t> saved_order;
    size_t saved_bytes = 0;
    static constexpr size_t SAVED_CAP = size_t(1) << 30;
    // admission: FIFO, or shortest predicted work first with aging
    int admission = SCGAL_ADMIT_FIFO;
    WorkModel model;
    static constexpr double AGE_MS = 1000.0;   // older queued requests go first, oldest first
    static constexpr size_t ADMIT_WINDOW = 256;

    // Index in the queue of the next request to admit (guarded by mu).
    size_t pick_next() const {
        if (admission == SCGAL_ADMIT_FIFO || queue.size() < 2) return 0;
        const double now = now_ms();
        if (now - queue.front().t_submit > AGE_MS) return 0;   // aged: the oldest first
        size_t best = 0;
        double bw = 0;
        const size_t lim = std::min(queue.size(), ADMIT_WINDOW);
        for (size_t k = 0; k < lim; ++k) {
            const Request& r = queue[k];
            const double work = r.predicted_iters * (double)std::max<long long>(r.nnz, r.n);
            if (k == 0 || work < bw) {
                best = k;
                bw = work;
            }
        }
        return best;
    }
    // batched engine state (device arrays owned by the worker thread)
    cudaStream_t bstream = nullptr;
    char* d_slots = nullptr;
    int* d_active = nullptr;
    int* d_ctl = nullptr;
    scgal::BatchLaunch* blaunch = nullptr;
    scgal::BatchStatus* d_status = nullptr;
    scgal::BatchStatus* h_status = nullptr;   // pinned
    std::vector<int> h_active;
    std::vector<unsigned char> slot_desc;     // host copy of one slot descriptor
    long long rounds = 0;

    bool init_batch() {
        if (bstream) return true;
        if (cudaStreamCreateWithFlags(&bstream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc(&d_slots, scgal::batch_slot_bytes() * (size_t)max_slots) != cudaSuccess ||
            cudaMalloc(&d_active, sizeof(int) * (size_t)max_slots) != cudaSuccess ||
            cudaMalloc(&d_ctl, sizeof(int) * scgal::BATCH_CTL_INTS) != cudaSuccess ||
            cudaMalloc(&d_status, sizeof(scgal::BatchStatus) * (size_t)max_slots) != cudaSuccess ||
            cudaMallocHost(&h_status, sizeof(scgal::BatchStatus) * (size_t)max_slots) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        slot_desc.resize(scgal::batch_slot_bytes());
        blaunch = scgal::batch_launch_create();
        return blaunch != nullptr;
    }

    void free_batch() {
        if (bstream) cudaStreamSynchronize(bstream);
        scgal::batch_launch_destroy(blaunch);
        blaunch = nullptr;
        if (d_slots) cudaFree(d_slots);
        if (d_active) cudaFree(d_active);
        if (d_ctl) cudaFree(d_ctl);
        if (d_status) cudaFree(d_status);
        if (h_status) cudaFreeHost(h_status);
        if (bstream) cudaStreamDestroy(bstream);
        bstream = nullptr;
        d_slots = nullptr;
        d_active = nullptr;
        d_ctl = nullptr;
        d_status = nullptr;
        h_status = nullptr;
    }

    // The solve in s ended (status; its last iteration record if st): retired later.
    void finish(Slot& s, int status, const scgal_stats* st) {
        s.fin = true;
        s.fin_status = status;
        s.fin_has_st = st != nullptr;
        if (st) s.fin_st = *st;
    }

    // The finished solve's iterate, kept for warm starts (oldest dropped past the cap).
    void keep(Slot& s) {
        Saved v;
        v.n = s.req.n;
        v.R = s.req.prm.R;
        v.prec = s.req.prm.precision;
        v.z.resize((size_t)s.req.n);
        v.y.resize((size_t)s.req.n);
        v.S.resize((size_t)s.req.n * s.req.prm.R);
        if (scgal_get_state(s.h, v.z.data(), v.y.data(), v.S.data(), v.sc) != SCGAL_OK) return;
        std::lock_guard<std::mutex> lk(mu);
        saved_bytes += v.bytes();
        saved[s.req.id] = std::move(v);
        saved_order.push_back(s.req.id);
        while (saved_bytes > SAVED_CAP && !saved_order.empty()) {
            auto it = saved.find(saved_order.front());
            if (it != saved.end()) {
                saved_bytes -= it->second.bytes();
                saved.erase(it);
            }
            saved_order.pop_front();
        }
    }

    // A warm start from a kept iterate (same n, R and precision): z, y, S, p and
    // tau as kept, t at a quarter of the kept t.  Returns the starting t (1: cold).
    long long warm_start(Slot& s) {
        const uint64_t from = (uint64_t)s.req.prm.warm_from;
        std::lock_guard<std::mutex> lk(mu);
        auto it = saved.find(from);
        if (it == saved.end()) return 1;
        const Saved& v = it->second;
        if (v.n != s.req.n || v.R != s.req.prm.R || v.prec != s.req.prm.precision) return 1;
        const long long t0 = std::max<long long>(1, (long long)v.sc[2] / 4);
        if (t0 > s.req.prm.T_max) return 1;
        const double sc[4] = {v.sc[0], v.sc[1], (double)t0, 0.0};
        if (scgal_set_state(s.h, v.z.data(), v.y.data(), v.S.data(), sc) != SCGAL_OK) return 1;
        return t0;
    }

    void retire(Slot& s) {
        s.fin = false;
        publish(s, s.fin_status, s.fin_has_st ? &s.fin_st : nullptr);
    }

    void publish(Slot& s, int status, const scgal_stats* st) {
        scgal_result r;
        std::memset(&r, 0, sizeof(r));
        r.status = status;
        r.n = s.req.n;
        r.first_t = s.req.first_t;
        r.predicted_iterations = s.req.predicted_iters;
        if (st) {
            r.iterations = (st->converged ? st->t - 1 : st->t) - (s.req.first_t - 1);
            r.relgap = st->relgap;
            r.infeas = st->infeas;
            r.objective = st->p;
        }
        if (status >= 0 && s.h) {
            std::vector<double> lam(s.req.prm.R), err(s.req.prm.R);
            int64_t cut = 0;
            const int rc = scgal_reconstruct(s.h, nullptr, lam.data(), err.data(), &cut);
            if (rc == SCGAL_OK) {
                r.best_cut = cut;
                r.lambda_max = lam[0];
            } else {
                r.status = rc;
            }
        }
        if (status >= 0 && s.h && s.req.kind == 0 && s.req.prm.keep_state) keep(s);
        const double t = now_ms();
        r.queue_ms = s.req.t_admit - s.req.t_submit;
        r.latency_ms = t - s.req.t_submit;
        if (s.h) scgal_destroy(s.h);
        s.h = nullptr;
        std::lock_guard<std::mutex> lk(mu);
        if (st && s.req.kind == 0 && s.req.first_t == 1 && status >= 0) model.add(s.req.n, s.req.nnz, r.iterations);
        done[s.req.id] = r;
        in_use -= s.req.footprint;
        s.active = false;
        --active;
        ++completed;
        cv_done.notify_all();
    }

    void run() {
        for (;;) {
            // 1. admission
            std::vector<int> fresh;
            {
                std::unique_lock<std::mutex> lk(mu);
                while (stopping && !queue.empty()) {   // stop admitting: queued requests end unsolved
                    scgal_result res;
                    std::memset(&res, 0, sizeof(res));
                    res.status = SCGAL_ESTATE;
                    res.n = queue.front().n;
                    done[queue.front().id] = res;
                    ++rejected;
                    queue.pop_front();
                    cv_done.notify_all();
                }
                if (active == 0 && queue.empty()) {
                    if (stopping) {
                        free_batch();
                        return;
                    }
                    cv_work.wait_for(lk, std::chrono::milliseconds(50));
                    continue;
                }
                for (int i = 0; i < max_slots && !queue.empty(); ++i) {
                    if (slots[i].active) continue;
                    const size_t qi = pick_next();
                    Request& r = queue[qi];
                    if (in_use + r.footprint > budget) {
                        if (active == 0 && r.footprint > budget) {   // can never fit: reject
                            scgal_result res;
                            std::memset(&res, 0, sizeof(res));
                            res.status = SCGAL_ENOMEM;
                            res.n = r.n;
                            done[r.id] = res;
                            ++rejected;
                            queue.erase(queue.begin() + (long)qi);
                            cv_done.notify_all();
                            --i;
                            continue;
                        }
                        break;
                    }
                    slots[i].req = std::move(r);
                    queue.erase(queue.begin() + (long)qi);
                    slots[i].active = true;
                    slots[i].h = nullptr;
                    in_use += slots[i].req.footprint;
                    peak = std::max(peak, in_use);
                    ++active;
                    ++admitted;
                    fresh.push_back(i);
                }
            }
            const bool batch_ok = init_batch();
            // 2. one stretch of every resident solve, all enqueued before any wait:
            //    small FP32 instances in the batched engine, the others on their own streams
            std::vector<int> live;
            std::vector<int> bvar[scgal::BATCH_NVAR];
            h_active.clear();
            ++rounds;
            for (int j = 0; j < max_slots; ++j) {
                const int i = (int)((j + rounds) % max_slots);   // rotating order: no slot always last
                Slot& s = slots[i];
                if (!s.active || !s.h || s.fin) continue;
                if (s.batched) {
                    bvar[s.variant].push_back(i);
                    continue;
                }
                const int rc = scgal::launch_iterations(s.h, s.h->t_next + CHUNK - 1);
                if (rc) finish(s, rc, nullptr);
                else live.push_back(i);
            }
            int counts[scgal::BATCH_NVAR];
            for (int v = 0; v < scgal::BATCH_NVAR; ++v) {
                counts[v] = (int)bvar[v].size();
                h_active.insert(h_active.end(), bvar[v].begin(), bvar[v].end());
            }
            int brc = SCGAL_OK;
            if (!h_active.empty()) {
                brc = cudaMemcpyAsync(d_active, h_active.data(), sizeof(int) * h_active.size(),
                                      cudaMemcpyHostToDevice, bstream) == cudaSuccess ? SCGAL_OK : SCGAL_ECUDA;
                if (!brc)
                    brc = scgal::launch_batch(blaunch, d_slots, d_active, counts, d_ctl, 1 << 30, BATCH_BUDGET_NS,
                                              d_status, bstream);
                if (!brc && cudaMemcpyAsync(h_status, d_status, sizeof(scgal::BatchStatus) * (size_t)max_slots,
                                            cudaMemcpyDeviceToHost, bstream) != cudaSuccess)
                    brc = SCGAL_ECUDA;
            }
            // 3. while the round runs: set up the new solves, retire the finished ones
            double t0 = now_ms();
            for (int i : fresh) {
                Slot& s = slots[i];
                s.req.t_admit = now_ms();
                const int rc = (s.req.kind == 1)
                                   ? scgal_create_phase(s.req.masks.data(), s.req.L, s.req.n, s.req.b.data(), 0.0,
                                                        &s.req.prm, &s.h)
                                   : scgal_create_maxcut(s.req.row_ptr.data(), s.req.col.data(),
                                                         s.req.has_w ? s.req.w.data() : nullptr, s.req.n, s.req.nnz,
                                                         0.0, &s.req.prm, &s.h);
                if (rc) {
                    s.h = nullptr;
                    finish(s, rc, nullptr);
                    continue;
                }
                if (s.req.kind == 0 && s.req.prm.warm_from) s.req.first_t = warm_start(s);
                // small FP32 instances join the batched engine (else, or if its set-up
                // fails, they run on the handle's own graphs)
                s.batched = batch_ok && scgal::batch_eligible(s.h) && !scgal::batch_prepare(s.h, slot_desc.data()) &&
                            cudaMemcpy(d_slots + slot_desc.size() * (size_t)i, slot_desc.data(), slot_desc.size(),
                                       cudaMemcpyHostToDevice) == cudaSuccess;
                if (s.batched) s.variant = scgal::batch_variant(slot_desc.data());
            }
            double t1 = now_ms();
            const double d_admit = t1 - t0;
            for (int i = 0; i < max_slots; ++i) {
                Slot& s = slots[i];
                if (s.active && s.fin) retire(s);
            }
            t0 = now_ms();
            const double d_retire = t0 - t1;
            // 4. wait for the round; mark the solves that finished in it
            if (!h_active.empty()) {
                if (!brc && cudaStreamSynchronize(bstream) != cudaSuccess) brc = SCGAL_ECUDA;
                for (int i : h_active) {
                    Slot& s = slots[i];
                    if (brc) {
                        finish(s, brc, nullptr);
                        continue;
                    }
                    scgal_stats st;
                    std::memset(&st, 0, sizeof(st));
                    int done = 0;
                    const int rr = scgal::batch_apply(s.h, h_status[i], &st, &done);
                    if (rr) finish(s, rr, nullptr);
                    else if (done) finish(s, h_status[i].converged ? SCGAL_OK : SCGAL_ENOTDONE, &st);
                }
            }
            for (int i : live) {
                Slot& s = slots[i];
                scgal_stats st;
                std::memset(&st, 0, sizeof(st));
                int conv = 0;
                const int rc = scgal::finish_iterations(s.h, &st, &conv);
                if (rc) finish(s, rc, nullptr);
                else if (conv) finish(s, SCGAL_OK, &st);
                else if (s.h->t_next > s.req.prm.T_max) finish(s, SCGAL_ENOTDONE, &st);
            }
            const double d_wait = now_ms() - t0;
            std::lock_guard<std::mutex> lk(mu);
            wait_ms += d_wait;
            admit_ms += d_admit;
            retire_ms += d_retire;
            ++rounds_done;
        }
    }
};

extern "C" {

int scgal_server_create(size_t hbm_budget, int32_t max_slots, scgal_srv_t* out) {
    if (!out || max_slots < 1 || max_slots > 256 || hbm_budget == 0) return SCGAL_EINVAL;
    scgal_server* s = new scgal_server();
    s->budget = hbm_budget;
    s->max_slots = max_slots;
    s->slots.resize(max_slots);
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return SCGAL_OK;
}

int scgal_server_set_admission(scgal_srv_t s, int32_t policy) {
    if (!s || (policy != SCGAL_ADMIT_FIFO && policy != SCGAL_ADMIT_SHORTEST_PREDICTED)) return SCGAL_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    s->admission = policy;
    return SCGAL_OK;
}

int scgal_submit(scgal_srv_t s, const int32_t* row_ptr, const int32_t* col, const double* w, int32_t n, int64_t nnz,
                 const scgal_params* params, uint64_t* ticket) {
    if (!s || !row_ptr || (nnz > 0 && !col) || !params || !ticket || n < 2 || nnz < 0) return SCGAL_EINVAL;
    if (params->T_max < 1 || params->R < 1 || params->R > SCGAL_RMAX) return SCGAL_EINVAL;
    Request r;
    r.n = n;
    r.nnz = nnz;
    r.prm = *params;
    r.row_ptr.resize((size_t)n + 1);
    r.col.resize((size_t)nnz);
    // the caller's buffers may be host or device memory
    if (cudaMemcpy(r.row_ptr.data(), row_ptr, sizeof(int32_t) * (n + 1), cudaMemcpyDefault) != cudaSuccess ||
        (nnz && cudaMemcpy(r.col.data(), col, sizeof(int32_t) * nnz, cudaMemcpyDefault) != cudaSuccess)) {
        cudaGetLastError();
        return SCGAL_ECUDA;
    }
    if (w) {
        r.has_w = true;
        r.w.resize((size_t)nnz);
        if (nnz && cudaMemcpy(r.w.data(), w, sizeof(double) * nnz, cudaMemcpyDefault) != cudaSuccess) {
            cudaGetLastError();
            return SCGAL_ECUDA;
        }
    }
    r.footprint = estimate_footprint(n, nnz, *params);
    r.t_submit = now_ms();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return SCGAL_ESTATE;
    if (s->queue.size() >= scgal_server::QUEUE_MAX) return SCGAL_EBUSY;
    r.predicted_iters = s->model.predict(n, nnz, params->T_max);
    r.id = s->next_id++;
    *ticket = r.id;
    ++s->submitted;
    s->queue.push_back(std::move(r));
    s->cv_work.notify_one();
    return SCGAL_OK;
}

int scgal_submit_phase(scgal_srv_t s, const double* masks, int32_t L, int32_t n, const double* b,
                       const scgal_params* params, uint64_t* ticket) {
    if (!s || !masks || !b || !params || !ticket || L < 1 || n < 16 || n > (1 << 20) || (n & (n - 1)))
        return SCGAL_EINVAL;
    if (params->T_max < 1 || params->R < 1 || params->R > SCGAL_RMAX || params->R > n) return SCGAL_EINVAL;
    Request r;
    r.kind = 1;
    r.n = n;
    r.L = L;
    r.prm = *params;
    const size_t d = (size_t)L * n;
    r.masks.resize(2 * d);
    r.b.resize(d);
    // the caller's buffers may be host or device memory
    if (cudaMemcpy(r.masks.data(), masks, sizeof(double) * 2 * d, cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(r.b.data(), b, sizeof(double) * d, cudaMemcpyDefault) != cudaSuccess) {
        cudaGetLastError();
        return SCGAL_ECUDA;
    }
    r.footprint = estimate_footprint_phase(n, L, *params);
    r.t_submit = now_ms();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return SCGAL_ESTATE;
    if (s->queue.size() >= scgal_server::QUEUE_MAX) return SCGAL_EBUSY;
    r.id = s->next_id++;
    *ticket = r.id;
    ++s->submitted;
    s->queue.push_back(std::move(r));
    s->cv_work.notify_one();
    return SCGAL_OK;
}

int scgal_poll(scgal_srv_t s, uint64_t ticket, scgal_result* out, int32_t timeout_ms) {
    if (!s || !out) return SCGAL_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] { return s->done.count(ticket) > 0; };
    if (timeout_ms < 0) s->cv_done.wait(lk, ready);
    else if (timeout_ms > 0) s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    auto it = s->done.find(ticket);
    if (it == s->done.end()) return SCGAL_ETIMEOUT;
    *out = it->second;
    s->done.erase(it);
    return SCGAL_OK;
}

int scgal_server_get_stats(scgal_srv_t s, scgal_server_stats* out) {
    if (!s || !out) return SCGAL_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->admitted = s->admitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->active = s->active;
    out->queued = (int32_t)s->queue.size();
    out->device_bytes_in_use = (int64_t)s->in_use;
    out->device_bytes_peak = (int64_t)s->peak;
    out->rounds = s->rounds_done;
    out->wait_ms = s->wait_ms;
    out->admit_ms = s->admit_ms;
    out->retire_ms = s->retire_ms;
    return SCGAL_OK;
}

int scgal_server_destroy(scgal_srv_t s) {
    if (!s) return SCGAL_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (auto& sl : s->slots)
        if (sl.h) scgal_destroy(sl.h);
    delete s;
    return SCGAL_OK;
}

}  // extern "C"
