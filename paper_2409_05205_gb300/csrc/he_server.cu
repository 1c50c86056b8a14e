// he_server.cu -- request loop for encrypted inferences (host code only).
//
// A server holds registered models (their layer banks stay resident on the
// device) and serves inference requests as they arrive.  A request carries
// the input ciphertexts of every layer of its model and receives the
// extracted outputs; its layer calls run in order, one after the other, as
// in the protocol where the client's non-linear step sits between layers
// (taken here as zero time).  A scheduler thread forms batches of up to
// max_batch requests waiting for the same (model, layer) -- continuous
// batching: while a batch of a layer runs, the requests that reach that
// layer wait and form its next batch, which is issued when the running one
// completes (or at once when max_batch of them wait); layers with nothing
// running are issued at once, oldest waiting request first -- and runs
// each batch on one of several streams: host->device copies, the layer as a
// one-call plan, device->host copies, then an event of the batch's lane that
// the scheduler polls (no host callbacks: the driver runs every stream's
// callbacks on one thread, one after another, and completions waited behind
// each other under load).  Device buffers ("lanes": the
// batch's inputs and outputs and the plan's workspace) are allocated under an
// HBM budget and reused.  A lane's size is known before anything is
// allocated, so device memory never exceeds the budget; when the budget is
// spent, idle lanes of other shapes are retired, and their memory is freed
// once no batch is in flight (cudaFree waits for the whole device, so
// freeing earlier would stall every stream); requests wait meanwhile.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <sys/prctl.h>

#include "he_internal.h"
#include <nvtx3/nvToolsExt.h>

namespace {

// polling period of the in-flight batches' events; the scheduler thread's
// timer slack is set to 1 us so that the sleep is about this long
constexpr int kPollUs = 5;

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct ModelLayer {
    he_filters_t f;
    size_t in_words, out_words;  // per ciphertext
};

struct Model {
    std::vector<ModelLayer> layers;
};

struct Req {
    uint64_t id;
    uint32_t model, layer = 0;
    std::vector<const uint32_t *> in;
    std::vector<uint32_t *> out;
    double t_arrive, t_layer;  // arrival; entry into the current layer's queue
    double t_launch = 0.0;     // the current layer's batch launch
    bool done = false, failed = false;
    double t_done = 0.0;
};

struct Lane {
    uint32_t model, layer, bucket;
    uint32_t *d_in = nullptr, *d_out = nullptr;
    he_plan_t plan = nullptr;
    cudaEvent_t done = nullptr;  // recorded after the batch's last copy
    size_t bytes = 0;
    bool busy = false;
};

struct Batch;

struct Server {
    he_server_config cfg;
    std::vector<Model> models;
    std::vector<cudaStream_t> streams;
    uint32_t next_stream = 0;

    std::mutex mu;  // everything below; the scheduler holds it across CUDA calls
    std::condition_variable cv_sched;  // a submission or a stop
    std::condition_variable cv_done;
    std::vector<Batch *> flight;       // launched batches, polled through their lane's event
    std::map<uint64_t, Req *> reqs;
    std::map<std::pair<uint32_t, uint32_t>, std::deque<Req *>> queues;  // (model, layer) -> waiting
    std::map<std::pair<uint32_t, uint32_t>, uint32_t> running;          // (model, layer) -> batches in flight
    std::vector<Batch *> failed_launch;
    std::vector<Lane *> lanes;
    std::vector<Lane *> retired;  // evicted idle lanes, counted in bytes_in_use until freed
    size_t bytes_in_use = 0, bytes_peak = 0;
    uint64_t next_id = 1, submitted = 0, finished = 0, batches = 0, batched_calls = 0, failed = 0;
    uint64_t evictions = 0, batch_hist[4] = {0, 0, 0, 0};
    uint32_t inflight = 0;
    std::vector<double> lat_layer, lat_net, lat_wait, lat_run;
    bool stop = false;
    char error[256] = {0};
    std::thread sched;
};

struct Batch {
    Server *s;
    Lane *lane;
    std::vector<Req *> reqs;
    bool ok;
};

// largest power of two <= n, at most max_batch
uint32_t bucket_of(uint32_t n, uint32_t max_batch) {
    uint32_t b = 1;
    while (b * 2 <= n && b * 2 <= max_batch) b *= 2;
    return b;
}

void free_lane(Server *s, Lane *l) {
    if (l->done) cudaEventDestroy(l->done);
    he_plan_destroy(l->plan);
    cudaFree(l->d_in);
    cudaFree(l->d_out);
    s->bytes_in_use -= l->bytes;
    delete l;
}

// Retires one idle lane (another shape's buffers and plan); false if none is
// idle.  Its bytes stay counted until free_retired releases them.
bool retire_idle_lane(Server *s) {
    for (size_t i = 0; i < s->lanes.size(); ++i) {
        Lane *l = s->lanes[i];
        if (l->busy) continue;
        s->retired.push_back(l);
        s->lanes.erase(s->lanes.begin() + (long)i);
        ++s->evictions;
        return true;
    }
    return false;
}

// Frees the retired lanes, only while no batch is in flight: cudaFree
// synchronizes the device, which then stalls nothing.
void free_retired(Server *s) {
    if (s->inflight != 0 || s->retired.empty()) return;
    for (Lane *l : s->retired) free_lane(s, l);
    s->retired.clear();
}

// a free lane for (model, layer, bucket), allocating one if the budget
// allows.  The lane's bytes (batch buffers plus its plan's workspace) are
// computed first; idle lanes of other shapes are retired until they fit,
// and nothing is allocated unless they do.  nullptr when none can be had
// now.  At model load (may_retire false) no lane is retired.  Called with
// s->mu held.
Lane *get_lane(Server *s, uint32_t model, uint32_t layer, uint32_t bucket, bool may_retire = true) {
    for (Lane *l : s->lanes)
        if (!l->busy && l->model == model && l->layer == layer && l->bucket == bucket) return l;
    const ModelLayer &ml = s->models[model].layers[layer];
    const size_t io = (ml.in_words + ml.out_words) * bucket * sizeof(uint32_t);
    he_layer_call c{ml.f, nullptr, HE_COEFF, nullptr, bucket};
    size_t ws = 0;
    if (he_plan_workspace_bytes(&c, 1, &ws) != HE_OK) return nullptr;
    const size_t need = io + ws;
    if (need > s->cfg.hbm_budget_bytes) return nullptr;
    while (may_retire && s->bytes_in_use + need > s->cfg.hbm_budget_bytes && retire_idle_lane(s)) {
    }
    if (s->bytes_in_use + need > s->cfg.hbm_budget_bytes) free_retired(s);
    if (s->bytes_in_use + need > s->cfg.hbm_budget_bytes) return nullptr;
    Lane *l = new (std::nothrow) Lane();
    if (!l) return nullptr;
    l->model = model;
    l->layer = layer;
    l->bucket = bucket;
    if (cudaMalloc(&l->d_in, ml.in_words * bucket * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&l->d_out, ml.out_words * bucket * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(l->d_in);
        cudaFree(l->d_out);
        delete l;
        return nullptr;
    }
    c.d_in = l->d_in;
    c.d_out = l->d_out;
    if (cudaEventCreateWithFlags(&l->done, cudaEventDisableTiming) != cudaSuccess ||
        he_plan_create(&c, 1, &l->plan) != HE_OK) {
        cudaGetLastError();
        if (l->done) cudaEventDestroy(l->done);
        cudaFree(l->d_in);
        cudaFree(l->d_out);
        delete l;
        return nullptr;
    }
    l->bytes = need;
    s->bytes_in_use += l->bytes;
    s->bytes_peak = std::max(s->bytes_peak, s->bytes_in_use);
    s->lanes.push_back(l);
    return l;
}

// issue one batch on a stream.  Called with s->mu held.
bool launch(Server *s, Lane *lane, std::vector<Req *> &rs) {
    nvtxRangePushA("he_server batch");  // one range per batch launch on the scheduler thread
    struct Pop {
        ~Pop() { nvtxRangePop(); }
    } pop;
    const ModelLayer &ml = s->models[lane->model].layers[lane->layer];
    cudaStream_t st = s->streams[s->next_stream++ % s->streams.size()];
    Batch *b = new (std::nothrow) Batch{s, lane, rs, true};
    if (!b) return false;
    bool ok = true;
    for (size_t j = 0; j < rs.size() && ok; ++j)
        ok = cudaMemcpyAsync(lane->d_in + j * ml.in_words, rs[j]->in[lane->layer], ml.in_words * sizeof(uint32_t),
                             cudaMemcpyHostToDevice, st) == cudaSuccess;
    ok = ok && he_plan_run(lane->plan, st) == HE_OK;
    for (size_t j = 0; j < rs.size() && ok; ++j)
        ok = cudaMemcpyAsync(rs[j]->out[lane->layer], lane->d_out + j * ml.out_words, ml.out_words * sizeof(uint32_t),
                             cudaMemcpyDeviceToHost, st) == cudaSuccess;
    ok = ok && cudaEventRecord(lane->done, st) == cudaSuccess;
    if (!ok) {
        // let what was issued drain, then fail the batch here
        cudaStreamSynchronize(st);
        cudaGetLastError();
        b->ok = false;
        s->failed_launch.push_back(b);
        snprintf(s->error, sizeof(s->error), "batch launch failed");
        return false;
    }
    const double t = now_ms();
    for (Req *r : rs) r->t_launch = t;
    s->flight.push_back(b);
    lane->busy = true;
    ++s->inflight;
    ++s->running[{lane->model, lane->layer}];
    ++s->batches;
    s->batched_calls += rs.size();
    ++s->batch_hist[rs.size() >= 8 ? 3 : (rs.size() >= 4 ? 2 : (rs.size() >= 2 ? 1 : 0))];
    return true;
}

void finish_batch(Server *s, Batch *b) {
    const double t = now_ms();
    if (b->lane->busy) {
        b->lane->busy = false;
        --s->inflight;
        --s->running[{b->lane->model, b->lane->layer}];
    }
    for (Req *r : b->reqs) {
        if (!b->ok) {
            r->failed = true;
            r->done = true;
            r->t_done = t;
            ++s->finished;
            ++s->failed;
            continue;
        }
        s->lat_layer.push_back(t - r->t_layer);
        s->lat_wait.push_back(r->t_launch - r->t_layer);
        s->lat_run.push_back(t - r->t_launch);
        if (++r->layer == s->models[r->model].layers.size()) {
            r->done = true;
            r->t_done = t;
            s->lat_net.push_back(t - r->t_arrive);
            ++s->finished;
        } else {
            r->t_layer = t;
            s->queues[{r->model, r->layer}].push_back(r);
        }
    }
    delete b;
}

void scheduler(Server *s) {
    cudaSetDevice(s->cfg.device);
    prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);  // 1 us: short polling sleeps stay short
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // completions first: they free lanes and move requests to their next
        // layer.  A batch is done when its lane's event is; an error there
        // fails the batch's requests.
        std::vector<Batch *> done;
        for (size_t i = 0; i < s->flight.size();) {
            Batch *b = s->flight[i];
            const cudaError_t q = cudaEventQuery(b->lane->done);
            if (q == cudaErrorNotReady) {
                ++i;
                continue;
            }
            if (q != cudaSuccess) {
                cudaGetLastError();
                b->ok = false;
                snprintf(s->error, sizeof(s->error), "batch failed on the device");
            }
            done.push_back(b);
            s->flight[i] = s->flight.back();
            s->flight.pop_back();
        }
        done.insert(done.end(), s->failed_launch.begin(), s->failed_launch.end());
        s->failed_launch.clear();
        for (Batch *b : done) finish_batch(s, b);
        if (!done.empty()) s->cv_done.notify_all();
        free_retired(s);
        if (s->stop && s->inflight == 0) break;
        // dispatch: oldest waiting request first, each batch from one queue;
        // a queue whose layer has a batch in flight keeps collecting
        // requests until it completes, unless a full batch waits
        bool progress = true;
        while (!s->stop && progress && s->inflight < s->cfg.max_inflight) {
            progress = false;
            std::deque<Req *> *best = nullptr;
            std::pair<uint32_t, uint32_t> key{0, 0};
            double oldest = 0.0;
            for (auto &kv : s->queues) {
                if (kv.second.empty()) continue;
                auto run = s->running.find(kv.first);
                if (run != s->running.end() && run->second > 0 && kv.second.size() < s->cfg.max_batch) continue;
                if (!best || kv.second.front()->t_layer < oldest) {
                    best = &kv.second;
                    key = kv.first;
                    oldest = kv.second.front()->t_layer;
                }
            }
            if (!best) break;
            const uint32_t bucket = bucket_of((uint32_t)best->size(), s->cfg.max_batch);
            Lane *lane = nullptr;
            for (uint32_t b = bucket; b >= 1 && !lane; b /= 2) lane = get_lane(s, key.first, key.second, b);
            if (!lane) break;  // budget spent and every lane busy: wait for a completion
            std::vector<Req *> rs;
            for (uint32_t j = 0; j < lane->bucket; ++j) {
                rs.push_back(best->front());
                best->pop_front();
            }
            launch(s, lane, rs);
            progress = true;
        }
        if (!s->failed_launch.empty()) continue;
        if (s->flight.empty()) {
            // nothing on the GPU: sleep until a submission (or a stop)
            s->cv_sched.wait_for(lk, std::chrono::milliseconds(1));
        } else {
            // batches in flight: poll again after a few microseconds, with the
            // lock released so that submissions and waits go through
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(kPollUs));
            lk.lock();
        }
    }
}

}  // namespace

struct he_server_s : Server {};

extern "C" {

he_status he_server_create(const he_server_config *cfg, he_server_t *out) {
    if (!cfg || !out) return he_fail(HE_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (cfg->max_batch == 0 || cfg->max_batch > 8 || (cfg->max_batch & (cfg->max_batch - 1)))
        return he_fail(HE_ERR_ARG, "max_batch must be 1, 2, 4 or 8");
    if (cfg->streams == 0 || cfg->streams > 32) return he_fail(HE_ERR_ARG, "streams must be 1..32");
    if (cfg->max_inflight == 0) return he_fail(HE_ERR_ARG, "max_inflight must be >= 1");
    if (cfg->hbm_budget_bytes == 0) return he_fail(HE_ERR_ARG, "hbm_budget_bytes must be > 0");
    he_server_s *s = new (std::nothrow) he_server_s();
    if (!s) return he_fail(HE_ERR_NOMEM, "server");
    s->cfg = *cfg;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(cfg->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return he_fail(HE_ERR_CUDA, "cannot select the server's device");
    }
    for (uint32_t i = 0; i < cfg->streams; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            cudaSetDevice(prev);
            delete s;
            return he_fail(HE_ERR_CUDA, "stream creation failed");
        }
        s->streams.push_back(st);
    }
    cudaSetDevice(prev);
    s->sched = std::thread(scheduler, s);
    *out = s;
    return HE_OK;
}

he_status he_server_add_model(he_server_t s, const he_filters_t *layers, uint32_t nlayers, uint32_t *model_id) {
    if (!s || !layers || !model_id || nlayers == 0) return he_fail(HE_ERR_ARG, "NULL argument or no layers");
    Model m;
    for (uint32_t i = 0; i < nlayers; ++i) {
        const he_filters_s *f = layers[i];
        if (!f) return he_fail(HE_ERR_ARG, "NULL layer");
        if (f->p->device != s->cfg.device) return he_fail(HE_ERR_ARG, "layer on another device");
        const size_t LN = (size_t)f->p->L * f->p->N;
        ModelLayer ml{layers[i], 0, 0};
        if (f->kind == HE_KIND_CONV) {
            ml.in_words = (size_t)f->lay.G * 2u * LN;
            ml.out_words = (size_t)f->lay.H * 2u * LN;
        } else {
            ml.in_words = 2u * LN;
            ml.out_words = (size_t)f->fl.P_fc * 2u * LN;
        }
        // a batch-1 lane (inputs, outputs and its plan's workspace) must fit
        // the budget, or the layer could never run
        he_layer_call c{layers[i], nullptr, HE_COEFF, nullptr, 1};
        size_t ws = 0;
        const he_status st = he_plan_workspace_bytes(&c, 1, &ws);
        if (st != HE_OK) return st;
        if ((ml.in_words + ml.out_words) * sizeof(uint32_t) + ws > s->cfg.hbm_budget_bytes)
            return he_fail(HE_ERR_ARG, "hbm_budget_bytes is too small for one of the model's layers");
        m.layers.push_back(ml);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    *model_id = (uint32_t)s->models.size();
    s->models.push_back(std::move(m));
    // lanes (batch buffers and plan) built now while the budget allows, so
    // that serving does not build them on the request path (a plan build
    // allocates and copies synchronously, stalling every stream): per layer
    // kLanesBatch1 of batch 1 -- requests of one model reach the same layer
    // at nearly the same time -- and one of every larger batch size
    constexpr uint32_t kLanesBatch1 = 3;
    std::vector<Lane *> held;  // built lanes are marked busy so get_lane builds new ones
    bool room = true;
    for (uint32_t b = 1; room && b <= s->cfg.max_batch; b *= 2)
        for (uint32_t i = 0; room && i < nlayers; ++i)
            for (uint32_t k = 0; room && k < (b == 1 ? std::min(kLanesBatch1, s->cfg.max_inflight) : 1u); ++k) {
                Lane *l = get_lane(s, *model_id, i, b, false);
                if (!l) {
                    room = false;  // budget reached: the rest on demand
                    break;
                }
                l->busy = true;
                held.push_back(l);
            }
    for (Lane *l : held) l->busy = false;
    return HE_OK;
}

he_status he_server_submit(he_server_t s, uint32_t model_id, const uint32_t *const *h_in, uint32_t *const *h_out,
                           uint64_t *ticket) {
    if (!s || !h_in || !h_out || !ticket) return he_fail(HE_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (model_id >= s->models.size()) return he_fail(HE_ERR_ARG, "unknown model");
    if (s->stop) return he_fail(HE_ERR_ARG, "server is stopping");
    const size_t nl = s->models[model_id].layers.size();
    for (size_t i = 0; i < nl; ++i)
        if (!h_in[i] || !h_out[i]) return he_fail(HE_ERR_ARG, "NULL layer buffer");
    Req *r = new (std::nothrow) Req();
    if (!r) return he_fail(HE_ERR_NOMEM, "request");
    r->id = s->next_id++;
    r->model = model_id;
    r->in.assign(h_in, h_in + nl);
    r->out.assign(h_out, h_out + nl);
    r->t_arrive = r->t_layer = now_ms();
    s->reqs[r->id] = r;
    s->queues[{model_id, 0}].push_back(r);
    ++s->submitted;
    *ticket = r->id;
    s->cv_sched.notify_one();
    return HE_OK;
}

he_status he_server_wait(he_server_t s, uint64_t ticket, uint32_t timeout_ms, he_request_stats *st) {
    if (!s) return he_fail(HE_ERR_ARG, "NULL argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return he_fail(HE_ERR_ARG, "unknown ticket");
    Req *r = it->second;
    if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [r] { return r->done; }))
        return he_fail(HE_ERR_TIMEOUT, "request not finished within the timeout");
    if (st) {
        st->arrive_ms = r->t_arrive;
        st->done_ms = r->t_done;
        st->latency_ms = r->t_done - r->t_arrive;
    }
    const bool failed = r->failed;
    s->reqs.erase(it);
    delete r;
    if (failed) return he_fail(HE_ERR_CUDA, "the request's batch failed");
    return HE_OK;
}

he_status he_server_report(he_server_t s, he_server_report_t *rep) {
    if (!s || !rep) return he_fail(HE_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    memset(rep, 0, sizeof(*rep));
    rep->submitted = s->submitted;
    rep->finished = s->finished;
    rep->failed = s->failed;
    rep->batches = s->batches;
    rep->batched_calls = s->batched_calls;
    rep->lanes = s->lanes.size();
    rep->bytes_in_use = s->bytes_in_use;
    rep->bytes_peak = s->bytes_peak;
    rep->evictions = s->evictions;
    for (int i = 0; i < 4; ++i) rep->batch_hist[i] = s->batch_hist[i];
    return HE_OK;
}

he_status he_server_latencies(he_server_t s, int which, double *out_ms, uint64_t cap, uint64_t *n) {
    if (!s || !n || which < 0 || which > 3) return he_fail(HE_ERR_ARG, "bad argument");
    std::lock_guard<std::mutex> lk(s->mu);
    const std::vector<double> &v =
        which == 0 ? s->lat_net : (which == 1 ? s->lat_layer : (which == 2 ? s->lat_wait : s->lat_run));
    *n = v.size();
    if (out_ms)
        for (size_t i = 0; i < v.size() && i < cap; ++i) out_ms[i] = v[i];
    return HE_OK;
}

void he_server_destroy(he_server_t s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // requests still queued never start; in-flight batches finish first
        for (auto &kv : s->queues) kv.second.clear();
        s->cv_sched.notify_one();
    }
    s->sched.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->cfg.device);
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (Lane *l : s->lanes) free_lane(s, l);
    for (Lane *l : s->retired) free_lane(s, l);
    for (auto &kv : s->reqs) delete kv.second;
    cudaSetDevice(prev);
    delete s;
}

}  // extern "C"
