// serve.cu -- request serving with continuous batching (host runtime).
//
// A server owns n_slots contexts, each with its own CUDA stream and one worker
// thread.  Requests wait in a FIFO queue; a free worker admits the head of the
// queue as soon as its estimated device footprint fits in what is left of
// the memory pool, so new requests enter while others are still running and
// the kernels of different slots overlap on the GPU.  A slot keeps its basis
// tables (shell pairs, Hermite coefficients, Schwarz diagonals) resident and
// skips the set-up when the next request carries the same basis.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "qdt_internal.cuh"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

int ncart_h(int l) { return (l + 1) * (l + 2) / 2; }

struct BasisCopy {
    std::vector<double> xyz, exps, coefs;
    std::vector<int> center, l, nprim;
    bool same(const qdt_request &r) const {
        if ((int)center.size() != r.n_shells || (int)xyz.size() != 3 * r.n_centers) return false;
        if (std::memcmp(xyz.data(), r.xyz, xyz.size() * sizeof(double))) return false;
        if (std::memcmp(center.data(), r.shell_center, center.size() * sizeof(int))) return false;
        if (std::memcmp(l.data(), r.shell_l, l.size() * sizeof(int))) return false;
        if (std::memcmp(nprim.data(), r.shell_nprim, nprim.size() * sizeof(int))) return false;
        long long np = 0;
        for (int s = 0; s < r.n_shells; ++s) np += r.shell_nprim[s];
        if ((long long)exps.size() != np) return false;
        return !std::memcmp(exps.data(), r.exps, np * sizeof(double)) &&
               !std::memcmp(coefs.data(), r.coefs, np * sizeof(double));
    }
    void set(const qdt_request &r) {
        xyz.assign(r.xyz, r.xyz + 3 * r.n_centers);
        center.assign(r.shell_center, r.shell_center + r.n_shells);
        l.assign(r.shell_l, r.shell_l + r.n_shells);
        nprim.assign(r.shell_nprim, r.shell_nprim + r.n_shells);
        long long np = 0;
        for (int s = 0; s < r.n_shells; ++s) np += r.shell_nprim[s];
        exps.assign(r.exps, r.exps + np);
        coefs.assign(r.coefs, r.coefs + np);
    }
};

struct Record {
    qdt_request r;
    size_t foot = 0;
    double t_submit = 0, t_done = 0;
    bool done = false;
    bool retried = false;       // ran out of memory beside other requests: runs again alone
    int status = QDT_OK;
    qdt_stats st{};
};

}  // namespace

struct qdt_server {
    int device = 0;
    size_t pool = 0, used = 0;
    int running = 0;            // requests admitted and not finished
    std::vector<qdt_ctx *> ctx;
    std::vector<BasisCopy> basis;
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Record> recs;
    uint64_t next = 1;
    bool stop = false;
};

namespace {

void worker(qdt_server *S, int slot) {
    cudaSetDevice(S->device);
    qdt_ctx *c = S->ctx[slot];
    for (;;) {
        uint64_t id = 0;
        qdt_request r;
        size_t foot = 0;
        bool others = false;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] {
                if (S->stop && S->queue.empty()) return true;
                if (S->queue.empty()) return false;
                const Record &h = S->recs[S->queue.front()];
                // a retried request waits until nothing else is admitted
                if (h.retried) return S->running == 0;
                return S->used + h.foot <= S->pool;
            });
            if (S->queue.empty()) return;
            id = S->queue.front();
            S->queue.pop_front();
            Record &rec = S->recs[id];
            r = rec.r;
            foot = rec.foot;
            S->used += foot;
            S->running++;
            others = S->running > 1;
        }
        int rc = QDT_OK;
        if (!S->basis[slot].same(r)) {
            rc = qdt_set_basis(c, r.n_centers, r.xyz, r.n_shells, r.shell_center, r.shell_l, r.shell_nprim,
                               r.exps, r.coefs);
            if (rc == QDT_OK) S->basis[slot].set(r);
            else S->basis[slot] = BasisCopy();
        }
        if (rc == QDT_OK) rc = qdt_set_coefficients(c, r.nK, r.CL, r.CS);
        qdt_stats st{};
        if (rc == QDT_OK)
            rc = qdt_transform(c, r.blocks, r.k_begin, r.k_end, r.schwarz_tau, r.precision, r.out, r.out_bytes, &st);
        // the footprint estimate counts one request per slot: drop this one's workspace
        qdt::release_workspace(c);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            Record &rec = S->recs[id];
            S->used -= foot;
            S->running--;
            if (rc == QDT_ERR_OOM && others && !rec.retried) {
                // device memory ran out beside other requests (the estimate is not a
                // bound): queue it first, to run again when nothing else is admitted
                rec.retried = true;
                S->queue.push_front(id);
            } else {
                rec.status = rc;
                rec.st = st;
                rec.t_done = now_s();
                rec.done = true;
            }
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

size_t qdt_footprint(const qdt_request *q) {
    if (!q || q->n_shells <= 0 || q->k_end <= q->k_begin) return 0;
    long long nL = 0, nsh = q->n_shells;
    double npp = 0;
    for (int s = 0; s < q->n_shells; ++s) {
        nL += ncart_h(q->shell_l[s]);
        npp += q->shell_nprim[s];
    }
    npp = (npp / nsh) * (npp / nsh);
    const double nS = 3.0 * nL, nKa = q->k_end - q->k_begin, nRS = nKa * (nKa + 1) / 2;
    const double M0 = nL * (nL + 1) / 2.0 + nS * (nS + 1) / 2.0, M1 = nL * nS;
    const double split = q->precision == QDT_SPLIT ? 1.0 : 0.0;
    double b = 0;
    auto wrows = [](double M, double mult) { return std::min(M * M * mult * mult * 8.0, 24.0 * (1u << 30)); };
    if (q->blocks & QDT_COULOMB) {
        double D = 8.0 * M0 * 4 * nRS;
        double W = wrows(M0, 1);
        b = std::max(b, 3 * D + W + split * (1.5 * W + 3 * 1.5 * D));
    }
    if (q->blocks & (QDT_GAUNT | QDT_GAUGE)) {
        double D = 8.0 * M1 * 12 * nRS;
        double W = wrows(M1, (q->blocks & QDT_GAUGE) ? 3 : 1) + ((q->blocks & QDT_GAUNT) ? wrows(M1, 1) : 0);
        b = std::max(b, 4 * D + W + split * (1.5 * W + 3 * 1.5 * D));
    }
    const double NO = 4 * nRS;
    b += 9.0 * NO * NO * 8;                                  // O + split-K partial sums
    b += 8.0 * (M0 + M1) * npp * 84;                         // Hermite coefficients
    b += 256.0 * (1 << 20);                                  // small tables
    return (size_t)b;
}

int qdt_server_create(qdt_server **out, int device, int n_slots, size_t pool_bytes) {
    if (!out || n_slots < 1 || n_slots > 16) return QDT_ERR_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return QDT_ERR_CUDA; }
    if (pool_bytes == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); return QDT_ERR_CUDA; }
        pool_bytes = (size_t)(0.8 * fr);
    }
    qdt_server *S = new (std::nothrow) qdt_server();
    if (!S) return QDT_ERR_OOM;
    S->device = device;
    S->pool = pool_bytes;
    for (int i = 0; i < n_slots; ++i) {
        qdt_ctx *c = nullptr;
        int rc = qdt_create(&c, device, nullptr);
        if (rc != QDT_OK) {
            for (qdt_ctx *x : S->ctx) qdt_destroy(x);
            delete S;
            return rc;
        }
        S->ctx.push_back(c);
    }
    S->basis.resize(n_slots);
    for (int i = 0; i < n_slots; ++i) S->workers.emplace_back(worker, S, i);
    *out = S;
    return QDT_OK;
}

void qdt_server_destroy(qdt_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto &t : S->workers) t.join();
    for (qdt_ctx *c : S->ctx) qdt_destroy(c);
    delete S;
}

int qdt_submit(qdt_server *S, const qdt_request *req, uint64_t *handle) {
    if (!S || !req || !handle) return QDT_ERR_ARG;
    if (req->n_shells <= 0 || req->nK <= 0 || req->k_begin < 0 || req->k_end > req->nK || req->k_end <= req->k_begin ||
        !req->out)
        return QDT_ERR_ARG;
    size_t foot = qdt_footprint(req);
    if (foot > S->pool) return QDT_ERR_ADMISSION;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        uint64_t id = S->next++;
        Record &rec = S->recs[id];
        rec.r = *req;
        rec.foot = foot;
        rec.t_submit = now_s();
        S->queue.push_back(id);
        *handle = id;
    }
    S->cv_work.notify_all();
    return QDT_OK;
}

int qdt_poll(qdt_server *S, uint64_t h, int *done) {
    if (!S || !done) return QDT_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->recs.find(h);
    if (it == S->recs.end()) return QDT_ERR_ARG;
    *done = it->second.done ? 1 : 0;
    return QDT_OK;
}

int qdt_wait(qdt_server *S, uint64_t h, double timeout_s, double *latency_s, qdt_stats *stats) {
    if (!S) return QDT_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->recs.find(h);
    if (it == S->recs.end()) return QDT_ERR_ARG;
    auto ready = [&] { return S->recs[h].done; };
    if (timeout_s < 0) {
        S->cv_done.wait(lk, ready);
    } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
        return QDT_ERR_TIMEOUT;
    }
    Record rec = S->recs[h];
    S->recs.erase(h);
    if (latency_s) *latency_s = rec.t_done - rec.t_submit;
    if (stats) *stats = rec.st;
    return rec.status;
}

}  // extern "C"
