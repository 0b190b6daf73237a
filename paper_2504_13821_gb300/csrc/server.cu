// Continuous-batching request server over the library's own entry points
// (trx_batched for small problems, trx_?trsm / trx_?trmm for the rest).
//
// Factors (triangular matrices on the device) are registered once and stay
// resident; requests name a factor, an operation, a side, alpha and a
// right-hand side, and are queued by trx_server_submit. Each
// trx_server_poll is one scheduling tick:
//   1. retire: launch groups whose completion event has fired release their
//      device-memory budget and in-flight slots, and their requests join the
//      completion queue;
//   2. admit: queued requests, oldest first, while the budget (right-hand
//      side bytes, plus the operand planes a tensor-core call uses) and the
//      slot count allow; admission does not wait for the device to drain;
//   3. launch: the admitted small problems (order <= small_k; FP64 ones up to
//      a work limit) go out as one
//      persistent batched launch per element type, the others one call each,
//      on the parallel stream with the least estimated cost in flight, one
//      handle (and workspace) per stream;
//   4. report: completed request ids and their status codes.
// The plan a request gets depends only on its own problem, never on what
// else is in flight, so a result is the same alone and in the mix.
//
// Request kinds: TRSM and TRMM in the factor's precision (trx_server_submit)
// and the refined FP32 TRSM (trx_server_submit_refined: FP32 factor and
// right-hand side, FP64 result, the FP32 solve plus a fixed number of
// float-float corrections, trx_strsm_refined_async, with no host read-back).
// FP64 TRMM requests: the recursive DFMA product or one float-float pass
// (config fp64_trmm).
// FP64 TRSM requests take the handles' FP64 engine (config fp64_corrections:
// the recursive DFMA solve, or the FP32 solve plus corrections).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <deque>
#include <vector>

#include "trx.h"

namespace trx {
const char* set_detail(const char* msg);   // the thread's error detail string (api.cu)
// swap a handle's workspace without synchronising the device: the caller
// has made sure no earlier work of the handle still runs (api.cu)
int handle_swap_workspace(trx_handle_t h, void* ptr, size_t bytes);
}

namespace {

constexpr int kServerMagic = 0x54525331;   // "TRS1"

int upc(char c) { return (c >= 'a' && c <= 'z') ? c - 'a' + 'A' : c; }

struct Fac {
    const void* A = nullptr;
    int64_t k = 0, lda = 1;
    char uplo = 'L', trans = 'N', diag = 'N';
    int elem = 4;
    int64_t outstanding = 0;   // submitted and not yet completed
    bool released = false;
    bool live = false;
};

struct Req {
    int64_t id;
    int fid;
    char op, side;          // op 'S', 'M', or 'R' (refined FP32 TRSM)
    double alpha;
    void* B;
    int64_t m, n, ldb;
    double* X = nullptr;    // refined: the FP64 result
    int64_t ldx = 0;
    cudaEvent_t ready;   // recorded on the caller's stream at submission
    size_t cost = 0;
};

struct Flight {
    cudaEvent_t done;
    uint64_t seq;                        // launch order across lanes
    double cost = 0;                     // its requests' estimated cost (stream choice)
    std::vector<int64_t> ids;
    std::vector<int> fids;
    size_t bytes;
};

}  // namespace

struct trx_server_s {
    int magic = kServerMagic;
    int device = 0;
    trx_server_config_t cfg{};
    std::vector<cudaStream_t> streams;
    std::vector<trx_handle_t> handles;
    std::vector<void*> ws;              // one workspace per handle (server-owned)
    std::vector<size_t> ws_bytes;
    cudaStream_t bstream = nullptr;     // batched launches
    trx_handle_t bhandle = nullptr;
    std::vector<Fac> facs;
    std::deque<Req> waiting;
    // launch groups in flight, one FIFO lane per stream (the large-request
    // streams, then the batched stream): a stream completes its work in
    // order, so retiring looks at lane fronts only and a poll costs
    // O(streams + completed), not O(in flight)
    std::vector<std::deque<Flight>> lanes;
    uint64_t flight_seq = 0;
    size_t inflight_bytes = 0;
    int64_t inflight_reqs = 0;
    std::deque<std::pair<int64_t, int>> done;   // (request id, status) not yet reported
    std::vector<cudaEvent_t> pool;
    int64_t next_id = 0;
    // estimated cost in flight per stream: k^2 n plus kLaunchCost for each
    // request (a request's fixed latency, in k^2 n units)
    std::vector<double> lane_cost;
};

namespace {

bool valid(trx_server_t s) { return s != nullptr && s->magic == kServerMagic; }

int fail(cudaError_t e, const char* what) {
    char buf[200];
    snprintf(buf, sizeof(buf), "server %s: %s", what, cudaGetErrorString(e));
    trx::set_detail(buf);
    return TRX_ERR_CUDA;
}

cudaError_t get_event(trx_server_t s, cudaEvent_t* ev) {
    if (!s->pool.empty()) {
        *ev = s->pool.back();
        s->pool.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
}
void put_event(trx_server_t s, cudaEvent_t ev) { s->pool.push_back(ev); }

// Whether a request goes to the batched launch. That kernel gives each
// problem one CTA; an FP64 problem of more than kSmallFp64Work (k^2 n) would
// hold its CTA for long on the slow FP64 pipe (about 0.15 ms at the limit),
// so it goes to the streams, whose engines spread it over the GPU.
constexpr double kSmallFp64Work = 1048576.0;
// A request's fixed latency (its launches, about 0.1-0.3 ms) in k^2 n units
// at the few TFLOP/s a latency-bound call reaches.
constexpr double kLaunchCost = 5e8;
bool is_small(const trx_server_s* s, const Req& r) {
    const Fac& f = s->facs[r.fid];
    if (f.k > s->cfg.small_k || r.op == 'R') return false;   // no refinement there
    const double nrhs = (double)(upc(r.side) == 'L' ? r.n : r.m);
    return f.elem == 4 || (double)f.k * (double)f.k * nrhs <= kSmallFp64Work;
}

// Device bytes a request holds while in flight: its right-hand side (and
// result), plus the operand planes of a tensor-core FP32 call (three BF16
// slices of the k x k triangle and of the k x nrhs right-hand side).
size_t cost_bytes(const trx_server_s* s, const Req& r) {
    const Fac& f = s->facs[r.fid];
    const int64_t nrhs = upc(r.side) == 'L' ? r.n : r.m;
    size_t b = (size_t)r.m * (size_t)r.n * (size_t)f.elem;
    if (r.op == 'R') b += (size_t)r.m * (size_t)r.n * 8;
    const bool tc_call = !is_small(s, r);
    const bool fp32_solve = f.elem == 4 || (upc(r.op) == 'S' && s->cfg.fp64_corrections > 0);
    if (tc_call && fp32_solve) b += 6 * (size_t)f.k * (size_t)(f.k + nrhs);
    return b;
}

// A request whose launch could not be issued completes at once with `code`.
void complete_now(trx_server_t s, const Req& r, int code) {
    s->done.emplace_back(r.id, code);
    s->facs[r.fid].outstanding -= 1;
    put_event(s, r.ready);
}

// Grow stream i's workspace. Only that stream is waited for (its handle's
// cached graphs point into the old buffer and are dropped); the buffers are
// stream-ordered allocations, so neither the allocation nor the release of
// the old one synchronises the device and the other streams keep running.
int ensure_ws(trx_server_t s, int i, size_t need) {
    if (need <= s->ws_bytes[i]) return TRX_SUCCESS;
    cudaStream_t st = s->streams[i];
    size_t bytes = std::max(need, s->ws_bytes[i] * 2);
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        bytes = need;
        if ((e = cudaMallocAsync(&p, bytes, st)) != cudaSuccess) {
            trx::set_detail("server workspace: cudaMallocAsync failed");
            return TRX_ERR_ALLOC;
        }
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) {
        cudaFreeAsync(p, st);
        return fail(e, "workspace swap");
    }
    const int rc = trx::handle_swap_workspace(s->handles[i], p, bytes);
    if (rc != TRX_SUCCESS) {
        cudaFreeAsync(p, st);
        return rc;
    }
    if (s->ws[i]) cudaFreeAsync(s->ws[i], st);
    s->ws[i] = p;
    s->ws_bytes[i] = bytes;
    return TRX_SUCCESS;
}

int launch_large(trx_server_t s, Req& r) {
    // the stream with the least estimated cost in flight: a request's cost is
    // its k^2 n plus a fixed term for its launches' latency, so neither a
    // large request nor a queue of small ones holds up what comes next
    int i = 0;
    for (int q = 1; q < (int)s->streams.size(); ++q)
        if (s->lane_cost[q] < s->lane_cost[i]) i = q;
    const Fac& f = s->facs[r.fid];
    const double cost = (double)f.k * (double)f.k * (double)(upc(r.side) == 'L' ? r.n : r.m) +
                        kLaunchCost;
    cudaStream_t st = s->streams[i];
    size_t need = 0;
    const char wop = r.op == 'R' ? 'S' : r.op;
    int rc = trx_workspace_size(s->handles[i], wop, r.side, r.m, r.n, f.elem, &need);
    if (rc == TRX_SUCCESS) rc = ensure_ws(s, i, need);
    if (rc != TRX_SUCCESS) return rc;
    cudaError_t e = cudaStreamWaitEvent(st, r.ready, 0);
    if (e != cudaSuccess) return fail(e, "wait");
    const bool trsm = upc(r.op) == 'S';
    if (r.op == 'R') {
        rc = trx_strsm_refined_async(s->handles[i], r.side, f.uplo, f.trans, f.diag, r.m, r.n,
                                     (float)r.alpha, static_cast<const float*>(f.A), f.lda,
                                     static_cast<const float*>(r.B), r.ldb, r.X, r.ldx,
                                     s->cfg.refine_corrections, st);
    } else if (f.elem == 4) {
        auto fn = trsm ? trx_strsm : trx_strmm;
        rc = fn(s->handles[i], r.side, f.uplo, f.trans, f.diag, r.m, r.n, (float)r.alpha,
                static_cast<const float*>(f.A), f.lda, static_cast<float*>(r.B), r.ldb, st);
    } else {
        auto fn = trsm ? trx_dtrsm : trx_dtrmm;
        rc = fn(s->handles[i], r.side, f.uplo, f.trans, f.diag, r.m, r.n, r.alpha,
                static_cast<const double*>(f.A), f.lda, static_cast<double*>(r.B), r.ldb, st);
    }
    if (rc != TRX_SUCCESS) {
        // part of the call may already be enqueued: the request's buffers
        // are idle before it is reported failed
        cudaStreamSynchronize(st);
        return rc;
    }
    Flight fl;
    // the launch is in flight: without a completion event, wait for it here
    // so the request's buffers are idle when it is reported failed
    if ((e = get_event(s, &fl.done)) != cudaSuccess) {
        cudaStreamSynchronize(st);
        return fail(e, "event");
    }
    if ((e = cudaEventRecord(fl.done, st)) != cudaSuccess) {
        put_event(s, fl.done);
        cudaStreamSynchronize(st);
        return fail(e, "record");
    }
    fl.ids.push_back(r.id);
    fl.fids.push_back(r.fid);
    fl.bytes = r.cost;
    put_event(s, r.ready);
    fl.seq = s->flight_seq++;
    fl.cost = cost;
    s->lane_cost[i] += cost;
    s->lanes[i].push_back(std::move(fl));
    s->inflight_reqs += 1;
    return TRX_SUCCESS;
}

int launch_small(trx_server_t s, std::vector<Req>& group, int elem) {
    std::vector<trx_problem_t> probs;
    probs.reserve(group.size());
    cudaError_t e;
    for (const Req& r : group) {
        if ((e = cudaStreamWaitEvent(s->bstream, r.ready, 0)) != cudaSuccess)
            return fail(e, "wait");
        const Fac& f = s->facs[r.fid];
        trx_problem_t p;
        p.op = r.op;
        p.side = r.side;
        p.uplo = f.uplo;
        p.transa = f.trans;
        p.diag = f.diag;
        p.m = r.m;
        p.n = r.n;
        p.alpha = r.alpha;
        p.A = f.A;
        p.lda = f.lda;
        p.B = r.B;
        p.ldb = r.ldb;
        probs.push_back(p);
    }
    int rc = trx_batched(s->bhandle, elem, (int64_t)probs.size(), probs.data(), s->bstream);
    if (rc != TRX_SUCCESS) {
        cudaStreamSynchronize(s->bstream);     // see launch_large
        return rc;
    }
    Flight fl;
    if ((e = get_event(s, &fl.done)) != cudaSuccess) {
        cudaStreamSynchronize(s->bstream);     // see launch_large
        return fail(e, "event");
    }
    if ((e = cudaEventRecord(fl.done, s->bstream)) != cudaSuccess) {
        put_event(s, fl.done);
        cudaStreamSynchronize(s->bstream);
        return fail(e, "record");
    }
    fl.bytes = 0;
    for (const Req& r : group) {
        fl.ids.push_back(r.id);
        fl.fids.push_back(r.fid);
        fl.bytes += r.cost;
        put_event(s, r.ready);
    }
    s->inflight_reqs += (int64_t)group.size();
    fl.seq = s->flight_seq++;
    s->lanes[s->lanes.size() - 1].push_back(std::move(fl));
    return TRX_SUCCESS;
}

// Retire finished launch groups; returns a CUDA error if a query failed.
int retire(trx_server_t s) {
    int first_err = TRX_SUCCESS;
    for (size_t li = 0; li < s->lanes.size(); ++li) {
        auto& lane = s->lanes[li];
        while (!lane.empty()) {
            Flight& fl = lane.front();
            const cudaError_t q = cudaEventQuery(fl.done);
            if (q == cudaErrorNotReady) break;
            const int status = q == cudaSuccess ? TRX_SUCCESS : fail(q, "launch group");
            if (status != TRX_SUCCESS && first_err == TRX_SUCCESS) first_err = status;
            for (size_t j = 0; j < fl.ids.size(); ++j) {
                s->done.emplace_back(fl.ids[j], status);
                s->facs[fl.fids[j]].outstanding -= 1;
            }
            s->inflight_bytes -= fl.bytes;
            s->inflight_reqs -= (int64_t)fl.ids.size();
            put_event(s, fl.done);
            if (li < s->lane_cost.size())
                s->lane_cost[li] = lane.size() == 1 ? 0.0 : s->lane_cost[li] - fl.cost;
            lane.pop_front();
        }
    }
    return first_err;
}

}  // namespace

extern "C" {

int trx_server_create(int device, const trx_server_config_t* config, trx_server_t* out) {
    if (!out) return TRX_ERR_INVALID_VALUE;
    *out = nullptr;
    trx_server_config_t cfg;
    cfg.streams = 4;
    cfg.small_k = TRX_BATCH_MAX_K;
    cfg.max_inflight = 4096;
    cfg.budget_bytes = (size_t)150 << 30;
    cfg.workspace_bytes = 0;
    cfg.graphs = 1;
    cfg.refine_corrections = 2;
    cfg.fp64_corrections = 0;
    cfg.fp64_trmm = 0;
    if (config) cfg = *config;
    if (cfg.streams < 1 || cfg.streams > 16 || cfg.small_k < 0 ||
        cfg.small_k > TRX_BATCH_MAX_K || cfg.max_inflight < 1 ||
        (cfg.graphs != 0 && cfg.graphs != 1) || cfg.refine_corrections < 0 ||
        cfg.refine_corrections > 16 || cfg.fp64_corrections < 0 || cfg.fp64_corrections > 16 ||
        (cfg.fp64_trmm != 0 && cfg.fp64_trmm != 1))
        return TRX_ERR_INVALID_VALUE;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(e, "cudaSetDevice");
    auto* s = new (std::nothrow) trx_server_s;
    if (!s) return TRX_ERR_ALLOC;
    s->device = device;
    s->cfg = cfg;
    s->lanes.resize((size_t)cfg.streams + 1);
    s->lane_cost.assign((size_t)cfg.streams, 0.0);
    int rc = TRX_SUCCESS;
    for (int i = 0; i < cfg.streams && rc == TRX_SUCCESS; ++i) {
        cudaStream_t st = nullptr;
        trx_handle_t h = nullptr;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) {
            rc = fail(e, "stream");
            break;
        }
        s->streams.push_back(st);
        if ((rc = trx_create(&h, device, 0)) != TRX_SUCCESS) break;
        s->handles.push_back(h);
        if ((rc = trx_set_option(h, TRX_OPT_GRAPH, cfg.graphs)) != TRX_SUCCESS) break;
        if ((rc = trx_set_option(h, TRX_OPT_FP64_TRSM, cfg.fp64_corrections)) != TRX_SUCCESS)
            break;
        if ((rc = trx_set_option(h, TRX_OPT_FP64_TRMM, cfg.fp64_trmm)) != TRX_SUCCESS) break;
        s->ws.push_back(nullptr);
        s->ws_bytes.push_back(0);
    }
    if (rc == TRX_SUCCESS) {
        if ((e = cudaStreamCreateWithFlags(&s->bstream, cudaStreamNonBlocking)) != cudaSuccess)
            rc = fail(e, "stream");
        else
            rc = trx_create(&s->bhandle, device, 0);
    }
    for (int i = 0; i < (int)s->handles.size() && rc == TRX_SUCCESS && cfg.workspace_bytes > 0;
         ++i)
        rc = ensure_ws(s, i, cfg.workspace_bytes);
    if (rc != TRX_SUCCESS) {
        trx_server_destroy(s);
        return rc;
    }
    *out = s;
    return TRX_SUCCESS;
}

int trx_server_destroy(trx_server_t s) {
    if (s == nullptr) return TRX_SUCCESS;
    if (!valid(s)) return TRX_ERR_HANDLE;
    cudaSetDevice(s->device);
    for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
    if (s->bstream) cudaStreamSynchronize(s->bstream);
    for (trx_handle_t h : s->handles) trx_destroy(h);
    if (s->bhandle) trx_destroy(s->bhandle);
    for (size_t i = 0; i < s->ws.size(); ++i)   // stream-ordered allocations
        if (s->ws[i]) cudaFreeAsync(s->ws[i], s->streams[i]);
    for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    if (s->bstream) cudaStreamDestroy(s->bstream);
    for (auto& lane : s->lanes)
        for (Flight& fl : lane) cudaEventDestroy(fl.done);
    for (Req& r : s->waiting) cudaEventDestroy(r.ready);
    for (cudaEvent_t ev : s->pool) cudaEventDestroy(ev);
    s->magic = 0;
    delete s;
    return TRX_SUCCESS;
}

int trx_server_register_factor(trx_server_t s, char uplo, char transa, char diag, int64_t k,
                               int elem_bytes, const void* A, int64_t lda, int* factor_id) {
    const int u = upc(uplo), t = upc(transa), d = upc(diag);
    if (u != 'L' && u != 'U') return -2;
    if (t != 'N' && t != 'T' && t != 'C') return -3;
    if (d != 'N' && d != 'U') return -4;
    if (k < 0) return -5;
    if (elem_bytes != 4 && elem_bytes != 8) return -6;
    if (k > 0 && A == nullptr) return -7;
    if (lda < std::max<int64_t>(1, k)) return -8;
    if (!factor_id) return -9;
    if (!valid(s)) return TRX_ERR_HANDLE;
    Fac f;
    f.A = A;
    f.k = k;
    f.lda = lda;
    f.uplo = (char)u;
    f.trans = (char)t;
    f.diag = (char)d;
    f.elem = elem_bytes;
    f.live = true;
    s->facs.push_back(f);
    *factor_id = (int)s->facs.size() - 1;
    return TRX_SUCCESS;
}

int trx_server_release_factor(trx_server_t s, int factor_id) {
    if (!valid(s)) return TRX_ERR_HANDLE;
    if (factor_id < 0 || factor_id >= (int)s->facs.size() || !s->facs[factor_id].live)
        return TRX_ERR_INVALID_VALUE;
    s->facs[factor_id].released = true;
    return TRX_SUCCESS;
}

int trx_server_submit(trx_server_t s, int factor_id, char op, char side, double alpha, void* B,
                      int64_t m, int64_t n, int64_t ldb, void* input_stream,
                      int64_t* request_id) {
    if (!valid(s)) return TRX_ERR_HANDLE;
    if (factor_id < 0 || factor_id >= (int)s->facs.size() || !s->facs[factor_id].live ||
        s->facs[factor_id].released)
        return -2;
    const int o = upc(op), sd = upc(side);
    if (o != 'S' && o != 'M') return -3;
    if (sd != 'L' && sd != 'R') return -4;
    const Fac& f = s->facs[factor_id];
    if (m < 0 || (sd == 'L' && m != f.k)) return -7;
    if (n < 0 || (sd == 'R' && n != f.k)) return -8;
    if (m > 0 && n > 0 && B == nullptr) return -6;
    if (ldb < std::max<int64_t>(1, m)) return -9;
    if (!request_id) return -11;
    Req r;
    r.id = s->next_id;
    r.fid = factor_id;
    r.op = (char)o;
    r.side = (char)sd;
    r.alpha = alpha;
    r.B = B;
    r.m = m;
    r.n = n;
    r.ldb = ldb;
    cudaError_t e = cudaSetDevice(s->device);
    if (e != cudaSuccess) return fail(e, "cudaSetDevice");
    if ((e = get_event(s, &r.ready)) != cudaSuccess) return fail(e, "event");
    if ((e = cudaEventRecord(r.ready, reinterpret_cast<cudaStream_t>(input_stream))) !=
        cudaSuccess) {
        put_event(s, r.ready);
        return fail(e, "record");
    }
    r.cost = cost_bytes(s, r);
    s->next_id += 1;
    s->facs[factor_id].outstanding += 1;
    s->waiting.push_back(r);
    *request_id = r.id;
    return TRX_SUCCESS;
}

int trx_server_submit_refined(trx_server_t s, int factor_id, char side, double alpha,
                              const void* B, int64_t m, int64_t n, int64_t ldb, double* X,
                              int64_t ldx, void* input_stream, int64_t* request_id) {
    if (!valid(s)) return TRX_ERR_HANDLE;
    if (factor_id < 0 || factor_id >= (int)s->facs.size() || !s->facs[factor_id].live ||
        s->facs[factor_id].released || s->facs[factor_id].elem != 4)
        return -2;
    const int sd = upc(side);
    if (sd != 'L' && sd != 'R') return -3;
    const Fac& f = s->facs[factor_id];
    if (m < 0 || (sd == 'L' && m != f.k)) return -7;
    if (n < 0 || (sd == 'R' && n != f.k)) return -8;
    if (m > 0 && n > 0 && B == nullptr) return -5;
    if (ldb < std::max<int64_t>(1, m)) return -9;
    if (m > 0 && n > 0 && X == nullptr) return -10;
    if (ldx < std::max<int64_t>(1, m)) return -11;
    if (!request_id) return -13;
    Req r;
    r.id = s->next_id;
    r.fid = factor_id;
    r.op = 'R';
    r.side = (char)sd;
    r.alpha = alpha;
    r.B = const_cast<void*>(B);
    r.m = m;
    r.n = n;
    r.ldb = ldb;
    r.X = X;
    r.ldx = ldx;
    cudaError_t e = cudaSetDevice(s->device);
    if (e != cudaSuccess) return fail(e, "cudaSetDevice");
    if ((e = get_event(s, &r.ready)) != cudaSuccess) return fail(e, "event");
    if ((e = cudaEventRecord(r.ready, reinterpret_cast<cudaStream_t>(input_stream))) !=
        cudaSuccess) {
        put_event(s, r.ready);
        return fail(e, "record");
    }
    r.cost = cost_bytes(s, r);
    s->next_id += 1;
    s->facs[factor_id].outstanding += 1;
    s->waiting.push_back(r);
    *request_id = r.id;
    return TRX_SUCCESS;
}

int trx_server_poll(trx_server_t s, int64_t* ids, int* status, int capacity, int* count) {
    if (!valid(s)) return TRX_ERR_HANDLE;
    if (!count || capacity < 0 || (capacity > 0 && (!ids || !status)))
        return TRX_ERR_INVALID_VALUE;
    *count = 0;
    cudaError_t e = cudaSetDevice(s->device);
    if (e != cudaSuccess) return fail(e, "cudaSetDevice");
    int first_err = retire(s);
    // admit, oldest first, while slots and budget allow
    std::vector<Req> small4, small8, large;
    while (!s->waiting.empty()) {
        Req& r = s->waiting.front();
        const int64_t admitted = (int64_t)(small4.size() + small8.size() + large.size());
        if (s->inflight_reqs + admitted >= s->cfg.max_inflight ||
            s->inflight_bytes + r.cost > s->cfg.budget_bytes) {
            // an oversized request alone on an idle server is admitted anyway
            if (!(s->inflight_reqs == 0 && admitted == 0)) break;
        }
        s->inflight_bytes += r.cost;
        const Fac& f = s->facs[r.fid];
        if (is_small(s, r))
            (f.elem == 4 ? small4 : small8).push_back(r);
        else
            large.push_back(r);
        s->waiting.pop_front();
    }
    auto fail_group = [&](std::vector<Req>& g, int rc) {
        for (Req& r : g) {
            s->inflight_bytes -= r.cost;
            complete_now(s, r, rc);
        }
        if (first_err == TRX_SUCCESS) first_err = rc;
    };
    if (!small4.empty()) {
        const int rc = launch_small(s, small4, 4);
        if (rc != TRX_SUCCESS) fail_group(small4, rc);
    }
    if (!small8.empty()) {
        const int rc = launch_small(s, small8, 8);
        if (rc != TRX_SUCCESS) fail_group(small8, rc);
    }
    for (Req& r : large) {
        const int rc = launch_large(s, r);
        if (rc != TRX_SUCCESS) {
            std::vector<Req> one{r};
            fail_group(one, rc);
        }
    }
    // release factors whose last request has completed
    for (Fac& f : s->facs)
        if (f.live && f.released && f.outstanding == 0) f.live = false;
    while (*count < capacity && !s->done.empty()) {
        ids[*count] = s->done.front().first;
        status[*count] = s->done.front().second;
        s->done.pop_front();
        *count += 1;
    }
    return first_err;
}

int trx_server_pending(trx_server_t s, int64_t* waiting, int64_t* inflight, int64_t* unreported) {
    if (!valid(s)) return TRX_ERR_HANDLE;
    if (waiting) *waiting = (int64_t)s->waiting.size();
    if (inflight) *inflight = s->inflight_reqs;
    if (unreported) *unreported = (int64_t)s->done.size();
    return TRX_SUCCESS;
}

int trx_server_wait(trx_server_t s) {
    if (!valid(s)) return TRX_ERR_HANDLE;
    cudaError_t e = cudaSetDevice(s->device);
    if (e != cudaSuccess) return fail(e, "cudaSetDevice");
    // the oldest launch group: waiting on it frees budget for the queue
    const Flight* oldest = nullptr;
    for (const auto& lane : s->lanes)
        if (!lane.empty() && (!oldest || lane.front().seq < oldest->seq)) oldest = &lane.front();
    if (oldest && (e = cudaEventSynchronize(oldest->done)) != cudaSuccess) return fail(e, "wait");
    return TRX_SUCCESS;
}

}  // extern "C"
