// Serving loop over the batch solver: continuous batching of independent
// solves (the request API of include/bddc.h).
//
// Host threads per server (kSetupThreads + 1):
//   setup threads take the queued requests in arrival order (consecutive
//                 requests with equal tol, at most max_batch), runs the
//                 setup of the batch (bddc::build_all, the dense local maps
//                 on the GPU), waits until the
//                 batch's device footprint fits the HBM budget beside the
//                 batches already admitted, uploads it (bddc::setup_from_packed)
//                 and hands it to the solve thread;
//   solve thread  runs the admitted batches one after another (one launch of
//                 the persistent kernel each), copies every request's slice
//                 of the results, frees the batch and returns its memory to
//                 the budget.
// While a batch is solved the next ones are set up and uploaded, and requests
// arriving meanwhile join a later batch.  Two setup threads work on two
// batches at once: the setup of a batch alternates between GPU-bound stages
// (the dense local maps and the face eigenproblems, FP64 on the device) and
// host-bound ones (constraints, correction maps, coarse inverse, packing), so
// one batch's host stages overlap the other's device stages.  Uploads use the
// legacy default stream with synchronous copies; solves run on the server's
// non-blocking stream, so they overlap on the device.  A batch that finishes
// its setup first is solved first; results are collected by ticket.
#include <cuda_runtime.h>

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

#include "bddc_internal.hpp"
#include "bddc_trace.hpp"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

int64_t cells_of(const bddc_grid& g) { return (int64_t)g.n[0] * g.n[1] * g.n[2]; }
int64_t faces_of(const bddc_grid& g) {
    int64_t f = (int64_t)(g.n[0] + 1) * g.n[1] * g.n[2] + (int64_t)g.n[0] * (g.n[1] + 1) * g.n[2];
    if (g.dim == 3) f += (int64_t)g.n[0] * g.n[1] * (g.n[2] + 1);
    return f;
}

struct Request {
    uint64_t ticket = 0;
    bddc_grid grid{};
    int perm_ncomp = 1;
    std::vector<double> perm, f, bc_value;
    std::vector<int32_t> part;
    std::vector<int8_t> bc_type;
    std::vector<int64_t> row_ptr, row_face;  // caller constraint rows (BDDC_CONSTRAINTS_EXPLICIT)
    std::vector<double> row_coef;
    double tol = 0.0;
    // result
    bool done = false;
    int status = BDDC_PENDING;
    std::vector<double> flux, pressure;
    bddc_stats stats{};
    bddc_request_info info{};
    Clock::time_point t_submit, t_setup;

    bddc_instance instance() const {
        bddc_instance in{};
        in.grid = grid;
        in.perm = perm.data();
        in.perm_ncomp = perm_ncomp;
        in.partition = part.data();
        in.bc_type = bc_type.data();
        if (row_ptr.size() > 1) {
            in.n_rows = (int)row_ptr.size() - 1;
            in.row_ptr = row_ptr.data();
            in.row_face = row_face.data();
            in.row_coef = row_coef.data();
        }
        return in;
    }
};
using ReqPtr = std::shared_ptr<Request>;

struct Batch {
    std::vector<ReqPtr> reqs;
    bddc_handle* h = nullptr;
    size_t bytes = 0;
    double tol = 0.0;
    int64_t id = 0;
};

// Device memory a batch's handle will hold, from its host setup: the
// uploaded arrays (the host arrays and their device forms have the same
// sizes, plus FP32-pair copies on the mixed path), the work vectors, the CG
// coefficient histories and the phase time stamps; 5 % and 1 MiB margin.
size_t estimate_device_bytes(const bddc::Packed& P, const bddc_options& opt, int n_inst) {
    auto bytes = [](const auto& v) { return v.size() * sizeof(v[0]); };
    size_t b = 0;
    b += bytes(P.inst_goff) * 14 + bytes(P.inst_vol) * 2;
    b += bytes(P.sub_inst) * 6 + bytes(P.off_S) * 9 + bytes(P.sub_d);
    b += bytes(P.slot_g) * 2 + bytes(P.slot_w) * 2 + bytes(P.slot_fcs) + bytes(P.cslot_n) + bytes(P.slot_coef);
    b += bytes(P.slot_fperm) + bytes(P.cslot_fstart) + bytes(P.slot_fcoefp) + bytes(P.cslot_c);
    b += bytes(P.cell_gid) + bytes(P.int_fid) + bytes(P.g_fid) + bytes(P.g_slot_a) * 2 + bytes(P.g_bsign);
    b += bytes(P.c_slot_a) * 2;
    b += bytes(P.S) + bytes(P.F64) + bytes(P.F32) + bytes(P.P64) + bytes(P.P32) + bytes(P.Gpre) + bytes(P.Gpost);
    b += bytes(P.Kinv) + 8 * (size_t)n_inst * (size_t)P.max_ncn;  // row padding
    const size_t gpost = bytes(P.Gpost) + 8 * (size_t)P.dev_Gpost_count;  // on the host or already on the device
    b += 8 * (size_t)P.dev_Gpost_count;
    if (opt.precision == BDDC_PREC_FP32) {
        b += gpost;                                   // G_post as FP32 pairs
        // weights, d*sigma and 1/n as FP32 pairs; coefficients as FP32
        b += bytes(P.slot_w) + bytes(P.slot_dsig) + bytes(P.cslot_n) * 2 + bytes(P.slot_coef) / 2 +
             bytes(P.slot_fcoefp) / 2;
    }
    const size_t G = (size_t)P.n_gamma, L = P.off_slot.empty() ? 0 : (size_t)P.off_slot.back();
    const size_t CL = P.off_cslot.empty() ? 0 : (size_t)P.off_cslot.back(), NS = (size_t)P.n_sub;
    b += 8 * (7 * G + 5 * L + CL + (size_t)P.n_coarse_vec + 12 * NS);
    b += 24 * (size_t)n_inst * ((size_t)opt.maxit + 1) + 64 * (size_t)n_inst;
    b += 16 * (16 + 4 * ((size_t)opt.maxit + 2));
    return b + b / 20 + (1u << 20);
}

}  // namespace

struct bddc_server {
    bddc_options opt{};
    size_t budget = 0;
    int max_batch = 1;
    int device = 0;
    cudaStream_t stream = nullptr;  // solves
    std::mutex mu;
    std::condition_variable cv;     // any change of the state below
    std::deque<ReqPtr> queue;       // submitted, not yet in a batch
    std::unordered_map<uint64_t, ReqPtr> reqs;  // submitted, not yet collected
    std::deque<Batch> ready;        // uploaded, waiting for the solve thread
    size_t in_use = 0, peak = 0;
    uint64_t next_ticket = 1;
    int64_t n_submitted = 0, n_completed = 0, n_failed = 0, n_batches = 0;
    int solving = 0;                // batches popped by the solve thread, not yet finished
    bool stop = false;
    static constexpr int kSetupThreads = 2;
    std::thread setup_thr[kSetupThreads], solve_thr;
};

namespace {

// mark a request done (caller holds no lock)
void finish(bddc_server* s, const ReqPtr& r, int status) {
    std::lock_guard<std::mutex> lk(s->mu);
    r->status = status;
    r->done = true;
    r->info.latency_ms = ms_between(r->t_submit, Clock::now());
    ++s->n_completed;
    if (status != BDDC_OK) ++s->n_failed;
    s->cv.notify_all();
}

void setup_batch(bddc_server* s, std::vector<ReqPtr> reqs) {
    const auto t0 = Clock::now();
    for (auto& r : reqs) {
        r->t_setup = t0;
        r->info.queue_ms = ms_between(r->t_submit, t0);
    }
    bddc::TraceStage stage("bddc_server: batch setup");
    std::vector<bddc_instance> inst;
    for (auto& r : reqs) inst.push_back(r->instance());
    bddc::Packed P;
    bddc::SetupResult res = bddc::build_all((int)inst.size(), inst.data(), s->opt, P, bddc::local_maps_device, bddc::face_eigen_device);
    if (res.code) {
        // find the failing requests: each alone; the others are set up again together
        std::vector<ReqPtr> ok;
        for (auto& r : reqs) {
            bddc::Packed Q;
            const bddc_instance one = r->instance();
            const bddc::SetupResult rr = bddc::build_all(1, &one, s->opt, Q, bddc::local_maps_device, bddc::face_eigen_device);
            if (rr.code) finish(s, r, rr.code);
            else ok.push_back(r);
        }
        if (ok.empty()) return;
        reqs.swap(ok);
        inst.clear();
        for (auto& r : reqs) inst.push_back(r->instance());
        P = bddc::Packed();
        res = bddc::build_all((int)inst.size(), inst.data(), s->opt, P, bddc::local_maps_device, bddc::face_eigen_device);
        if (res.code) {
            for (auto& r : reqs) finish(s, r, res.code);
            return;
        }
    }
    const int n = (int)reqs.size();
    const size_t need = estimate_device_bytes(P, s->opt, n);
    if (need > s->budget && n > 1) {
        // too large for the budget as one batch: two smaller batches
        std::vector<ReqPtr> second(reqs.begin() + n / 2, reqs.end());
        reqs.resize(n / 2);
        P = bddc::Packed();
        setup_batch(s, std::move(reqs));
        setup_batch(s, std::move(second));
        return;
    }
    {
        std::unique_lock<std::mutex> lk(s->mu);
        if (need > s->budget) {
            lk.unlock();
            for (auto& r : reqs) finish(s, r, BDDC_E_OOM);
            return;
        }
        s->cv.wait(lk, [&] { return s->stop || s->in_use + need <= s->budget; });
        if (s->stop) {
            lk.unlock();
            for (auto& r : reqs) finish(s, r, BDDC_E_INVALID_ARG);
            return;
        }
        s->in_use += need;
        s->peak = std::max(s->peak, s->in_use);
    }
    bddc_handle* h = nullptr;
    stage.next("bddc_server: upload");
    const int rc = bddc::setup_from_packed(n, s->opt, s->stream, std::move(P), &h);
    if (rc) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->in_use -= need;
            s->cv.notify_all();
        }
        for (auto& r : reqs) finish(s, r, rc);
        return;
    }
    const auto t1 = Clock::now();
    for (auto& r : reqs) r->info.setup_ms = ms_between(t0, t1);
    Batch b;
    b.reqs = std::move(reqs);
    b.h = h;
    b.tol = b.reqs.front()->tol;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        // account the handle's actual memory from now on
        const size_t actual = bddc::handle_device_bytes(h);
        s->in_use = s->in_use - need + actual;
        s->peak = std::max(s->peak, s->in_use);
        b.bytes = actual;
        b.id = s->n_batches++;
        s->ready.push_back(std::move(b));
        s->cv.notify_all();
    }
}

void setup_loop(bddc_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<ReqPtr> take;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return s->stop || !s->queue.empty(); });
            if (s->stop) return;
            const double tol = s->queue.front()->tol;
            while (!s->queue.empty() && (int)take.size() < s->max_batch && s->queue.front()->tol == tol) {
                take.push_back(s->queue.front());
                s->queue.pop_front();
            }
        }
        setup_batch(s, std::move(take));
    }
}

void solve_batch(bddc_server* s, Batch& b) {
    const auto t0 = Clock::now();
    const int n = (int)b.reqs.size();
    std::vector<int64_t> cell_off(n + 1, 0), face_off(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        cell_off[i + 1] = cell_off[i] + cells_of(b.reqs[i]->grid);
        face_off[i + 1] = face_off[i] + faces_of(b.reqs[i]->grid);
    }
    std::vector<double> f((size_t)cell_off[n]), bc((size_t)face_off[n]);
    for (int i = 0; i < n; ++i) {
        std::copy(b.reqs[i]->f.begin(), b.reqs[i]->f.end(), f.begin() + cell_off[i]);
        std::copy(b.reqs[i]->bc_value.begin(), b.reqs[i]->bc_value.end(), bc.begin() + face_off[i]);
    }
    for (auto& r : b.reqs) {  // the inputs are no longer needed: set up, and copied for the solve
        std::vector<double>().swap(r->perm);
        std::vector<double>().swap(r->f);
        std::vector<double>().swap(r->bc_value);
        std::vector<int32_t>().swap(r->part);
        std::vector<int8_t>().swap(r->bc_type);
        std::vector<int64_t>().swap(r->row_ptr);
        std::vector<int64_t>().swap(r->row_face);
        std::vector<double>().swap(r->row_coef);
    }
    std::vector<double> flux((size_t)face_off[n]), pres((size_t)cell_off[n]);
    std::vector<int> its(n, 0);
    bddc::TraceStage stage("bddc_server: batch solve");
    const int rc = bddc_solve(b.h, f.data(), bc.data(), b.tol, flux.data(), pres.data(), its.data());
    std::vector<int> status(n, rc);
    for (int i = 0; i < n; ++i) {
        Request& r = *b.reqs[i];
        if (rc == BDDC_OK || rc == BDDC_E_NOT_CONVERGED || rc == BDDC_E_BREAKDOWN) {
            // per-instance status: one instance's failure is not the others'
            bddc_get_stats(b.h, i, &r.stats);
            status[i] = r.stats.status;
            r.flux.assign(flux.begin() + face_off[i], flux.begin() + face_off[i + 1]);
            r.pressure.assign(pres.begin() + cell_off[i], pres.begin() + cell_off[i + 1]);
        }
    }
    bddc_destroy(b.h);
    b.h = nullptr;
    const auto t1 = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    s->in_use -= b.bytes;
    for (int i = 0; i < n; ++i) {
        Request& r = *b.reqs[i];
        r.info.solve_ms = ms_between(t0, t1);
        r.info.batch_size = n;
        r.info.batch_id = b.id;
        r.info.latency_ms = ms_between(r.t_submit, t1);
        r.status = status[i];
        r.done = true;
        ++s->n_completed;
        if (status[i] != BDDC_OK) ++s->n_failed;
    }
    s->cv.notify_all();
}

void solve_loop(bddc_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        Batch b;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return !s->ready.empty() || (s->stop && s->solving == 0); });
            if (s->ready.empty()) return;  // stopping and nothing admitted is left
            b = std::move(s->ready.front());
            s->ready.pop_front();
            ++s->solving;
        }
        solve_batch(s, b);
        std::lock_guard<std::mutex> lk(s->mu);
        --s->solving;
        s->cv.notify_all();
    }
}

}  // namespace

extern "C" {

int bddc_server_create(const bddc_options* opt_in, size_t hbm_budget_bytes, int max_batch, bddc_server** out) {
    if (!out) return BDDC_E_INVALID_ARG;
    *out = nullptr;
    if (hbm_budget_bytes == 0 || max_batch < 1) return BDDC_E_INVALID_ARG;
    bddc_options opt;
    bddc_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (!bddc::options_valid(opt)) return BDDC_E_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return BDDC_E_CUDA;
    }
    bddc_server* s = new bddc_server();
    s->opt = opt;
    s->budget = hbm_budget_bytes;
    s->max_batch = max_batch;
    cudaGetDevice(&s->device);
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return BDDC_E_CUDA;
    }
    for (std::thread& t : s->setup_thr) t = std::thread(setup_loop, s);
    s->solve_thr = std::thread(solve_loop, s);
    *out = s;
    return BDDC_OK;
}

int bddc_submit(bddc_server* s, const bddc_instance* inst, const double* f, const double* bc_value, double tol,
                uint64_t* ticket) {
    if (!s || !inst || !f || !bc_value || !ticket || !(tol > 0.0)) return BDDC_E_INVALID_ARG;
    const bddc_grid& g = inst->grid;
    if ((g.dim != 2 && g.dim != 3) || g.n[0] < 1 || g.n[1] < 1 || g.n[2] < 1 || (g.dim == 2 && g.n[2] != 1))
        return BDDC_E_INVALID_ARG;
    if (!inst->perm || !inst->partition || !inst->bc_type || (inst->perm_ncomp != 1 && inst->perm_ncomp != g.dim))
        return BDDC_E_INVALID_ARG;
    const int64_t nc = cells_of(g), nf = faces_of(g);
    if (nc > ((int64_t)1 << 30)) return BDDC_E_INVALID_ARG;
    auto r = std::make_shared<Request>();
    r->grid = g;
    r->perm_ncomp = inst->perm_ncomp;
    r->perm.assign(inst->perm, inst->perm + nc * inst->perm_ncomp);
    r->part.assign(inst->partition, inst->partition + nc);
    r->bc_type.assign(inst->bc_type, inst->bc_type + nf);
    if (inst->n_rows < 0) return BDDC_E_INVALID_ARG;
    if (inst->n_rows > 0) {
        if (!inst->row_ptr || !inst->row_face || !inst->row_coef) return BDDC_E_INVALID_ARG;
        r->row_ptr.assign(inst->row_ptr, inst->row_ptr + inst->n_rows + 1);
        const int64_t nnz = r->row_ptr.back();
        if (r->row_ptr[0] != 0 || nnz < 0) return BDDC_E_INVALID_ARG;
        for (int q = 0; q < inst->n_rows; ++q)
            if (r->row_ptr[q + 1] < r->row_ptr[q]) return BDDC_E_INVALID_ARG;
        r->row_face.assign(inst->row_face, inst->row_face + nnz);
        r->row_coef.assign(inst->row_coef, inst->row_coef + nnz);
    }
    r->f.assign(f, f + nc);
    r->bc_value.assign(bc_value, bc_value + nf);
    r->tol = tol;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return BDDC_E_INVALID_ARG;
    r->ticket = s->next_ticket++;
    s->reqs[r->ticket] = r;
    s->queue.push_back(r);
    ++s->n_submitted;
    *ticket = r->ticket;
    s->cv.notify_all();
    return BDDC_OK;
}

int bddc_poll(bddc_server* s, uint64_t ticket, double* flux, double* pressure, int* iterations, bddc_stats* stats,
              bddc_request_info* info) {
    if (!s) return BDDC_E_INVALID_ARG;
    ReqPtr r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return BDDC_E_INVALID_ARG;
        if (!it->second->done) return BDDC_PENDING;
        r = it->second;
        s->reqs.erase(it);
    }
    if (flux && !r->flux.empty()) std::copy(r->flux.begin(), r->flux.end(), flux);
    if (pressure && !r->pressure.empty()) std::copy(r->pressure.begin(), r->pressure.end(), pressure);
    if (iterations) *iterations = r->stats.iterations;
    if (stats) *stats = r->stats;
    if (info) *info = r->info;
    return r->status;
}

int bddc_wait(bddc_server* s, uint64_t ticket, double timeout_s) {
    if (!s) return BDDC_E_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return BDDC_E_INVALID_ARG;
    ReqPtr r = it->second;
    auto pred = [&] { return r->done; };
    if (timeout_s < 0) {
        s->cv.wait(lk, pred);
        return BDDC_OK;
    }
    return s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), pred) ? BDDC_OK : BDDC_PENDING;
}

int bddc_server_get_info(bddc_server* s, bddc_server_info* info) {
    if (!s || !info) return BDDC_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    info->submitted = s->n_submitted;
    info->completed = s->n_completed;
    info->failed = s->n_failed;
    info->batches = s->n_batches;
    info->device_bytes_in_use = s->in_use;
    info->device_bytes_peak = s->peak;
    return BDDC_OK;
}

void bddc_server_destroy(bddc_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->queue.clear();
        s->cv.notify_all();
    }
    for (std::thread& t : s->setup_thr)
        if (t.joinable()) t.join();
    if (s->solve_thr.joinable()) s->solve_thr.join();
    for (Batch& b : s->ready)  // admitted after the solve thread stopped: not solved
        if (b.h) bddc_destroy(b.h);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
