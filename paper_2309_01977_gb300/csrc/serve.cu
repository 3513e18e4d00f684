// Continuous-batching reconstruction server (spect_serve_*).
//
// Requests (geometry, mu, counts, iteration budget) arrive at any time and
// wait in a FIFO queue.  The device work happens in slots: a slot holds, for
// one acquisition geometry, a plan (geometry tables, attenuation cache,
// sensitivities), the image, counts and scatter buffers, a stream and a CUDA
// graph of one OSEM iteration (all subsets) captured once.  A scheduler
// thread admits a request into an idle slot of its geometry, or into a new
// slot when the slot fits the HBM budget (idle slots of other geometries are
// released to make room; later, smaller requests may pass a head that does
// not fit yet).  Admission uploads the request's counts and mu, recomputes
// the slot's attenuation cache and sensitivities, sets x = 1 and replays the
// iteration graph n_iters times, then reads the image back into pinned
// memory.  Slots on different streams overlap on the device; every kernel of
// a request reads and writes only its slot, so a result is bitwise the same
// alone or in any mix.  Latency is measured from submit to completion.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "internal.h"
#include "spect_serve.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_ms()
{
    return std::chrono::duration<double, std::milli>(Clock::now().time_since_epoch()).count();
}

// Pinned host buffers reused across requests (allocating pinned memory per
// request would stall the scheduler).
class PinnedPool {
public:
    ~PinnedPool()
    {
        for (auto& b : bufs_) cudaFreeHost(b.ptr);
    }
    float* take(size_t floats)
    {
        std::lock_guard<std::mutex> g(m_);
        for (auto& b : bufs_)
            if (!b.used && b.floats >= floats) {
                b.used = true;
                return b.ptr;
            }
        void* p = nullptr;
        if (cudaHostAlloc(&p, floats * sizeof(float), cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        bufs_.push_back({static_cast<float*>(p), floats, true});
        return static_cast<float*>(p);
    }
    void give(float* p)
    {
        if (!p) return;
        std::lock_guard<std::mutex> g(m_);
        for (auto& b : bufs_)
            if (b.ptr == p) b.used = false;
    }

private:
    struct Buf {
        float* ptr;
        size_t floats;
        bool used;
    };
    std::mutex m_;
    std::vector<Buf> bufs_;
};

struct Request {
    uint64_t id = 0;
    spect_geom geom{};
    std::vector<double> angles;
    std::vector<float> offsets;  // non-circular orbit, or empty
    std::vector<float> shifts;   // T_trans per angle, or empty
    std::vector<float> fov;      // T_fov weights, or empty
    float s = 0.f;
    int n_iters = 0;
    uint64_t tag = 0;
    size_t vol = 0, proj = 0, bytes = 0;
    float* h_mu = nullptr;  // pinned copies of the inputs, then the result
    float* h_y = nullptr;
    float* h_x = nullptr;
    int state = SPECT_REQ_QUEUED;
    int status = SPECT_OK;
    bool cancel = false;
    double t_submit = 0, t_admit = 0, t_done = 0;
    struct Slot* slot = nullptr;  // while admitted
};

// Device state for one acquisition geometry, reused by successive requests.
struct Slot {
    spect_geom geom{};
    std::vector<double> angles;
    std::vector<float> offsets, shifts, fov;
    spect_plan* plan = nullptr;
    float* d_mu = nullptr;
    float* d_y = nullptr;
    float* d_x = nullptr;
    float* d_s = nullptr;
    size_t vol = 0, proj = 0, bytes = 0;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t iter = nullptr;  // one OSEM iteration (all subsets); NULL: launch directly
    cudaEvent_t done = nullptr;
    bool busy = false;
    bool fresh = false;  // plan built from the current request's mu
    Request* req = nullptr;
};

bool same_geometry(const Slot& sl, const Request& r)
{
    const spect_geom &a = sl.geom, &b = r.geom;
    return a.nx == b.nx && a.ny == b.ny && a.nz == b.nz && a.voxel_cm == b.voxel_cm && a.n_angles == b.n_angles &&
           a.psf_sigma0 == b.psf_sigma0 && a.psf_slope == b.psf_slope && a.psf_nsigma == b.psf_nsigma &&
           a.det_offset == b.det_offset && a.n_subsets == b.n_subsets && a.flags == b.flags &&
           sl.angles == r.angles && sl.offsets == r.offsets && sl.shifts == r.shifts && sl.fov == r.fov;
}

}  // namespace

struct spect_server {
    spect_serve_cfg cfg{};
    int device = 0;
    int num_sms = 0;
    std::mutex m;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::vector<Request*> active;
    std::vector<Slot*> slots;
    std::map<uint64_t, Request*> all;
    std::vector<cudaStream_t> streams;
    size_t next_stream = 0;
    size_t in_use = 0;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread worker;
    PinnedPool pinned;
    spect_serve_stats stats{};
    std::vector<double> latencies;
    double t_first_submit = -1, t_last_done = 0;
};

namespace {

// Upper bound of a slot's device memory: the plan plus image, counts, mu.
size_t request_bytes(const spect_geom& g, int num_sms)
{
    const size_t n = (size_t)g.nx, nz = (size_t)g.nz, na = (size_t)g.n_angles, M = (size_t)g.n_subsets;
    const size_t vol = n * n * nz, plane = n * nz;
    const size_t max_subset = (na + M - 1) / M;
    size_t b = 0;
    b += M * vol * 4;                                                    // sensitivities
    b += std::max<size_t>(4 * (size_t)num_sms, max_subset) * plane * 4;  // depth-chunk partials
    b += na * (n + 7) * (n + 7) * spect::kMaxCand * 8;                   // gather tables (either layout)
    b += na * ((n + 3) / 4) * ((n + 3) / 4) * spect::kFpDescInts * 4;    // tiled-gather footprints
    b += std::max<size_t>(max_subset, 16) * vol * 4;                     // rotated-frame volumes
    b += max_subset * plane * 4 + vol * 4;                               // ratio, back projection
    if (g.flags & SPECT_FLAG_ATTEN) b += na * vol * 4;                   // attenuation cache
    const size_t tables = g.det_offsets ? na : 1;                        // PSF tables (orbit)
    if (g.flags & SPECT_FLAG_PSF_BF16) b += tables * n * 2 * 128 * 128 * 2;  // Toeplitz tiles (hi, lo)
    b += tables * (n * 41 * 4 + spect::psf_int_stride((int)n) * 4);             // taps, radii, work, chunk bounds
    if (g.fov_mask) b += na * plane * 4;                                 // T_fov weights
    b += 3 * vol * 4 + na * plane * 4;                                   // mu, x, y
    b += 1 << 20;                                                        // tables, small scratch
    return b;
}

void destroy_slot(Slot* sl)
{
    if (sl->done) cudaEventSynchronize(sl->done);  // an idle slot's last work has completed
    if (sl->iter) cudaGraphExecDestroy(sl->iter);
    if (sl->done) cudaEventDestroy(sl->done);
    if (sl->plan) spect_plan_destroy(sl->plan);
    if (sl->d_mu) cudaFree(sl->d_mu);
    if (sl->d_y) cudaFree(sl->d_y);
    if (sl->d_x) cudaFree(sl->d_x);
    if (sl->d_s) cudaFree(sl->d_s);
    delete sl;
}

// A new slot for r's geometry, its plan built from r's mu.  Called without
// the lock.
int create_slot(spect_server* sv, Request* r, cudaStream_t st, Slot** out)
{
    Slot* sl = new (std::nothrow) Slot();
    if (!sl) return SPECT_ENOMEM;
    sl->geom = r->geom;
    sl->angles = r->angles;
    sl->offsets = r->offsets;
    sl->shifts = r->shifts;
    sl->fov = r->fov;
    sl->vol = r->vol;
    sl->proj = r->proj;
    sl->bytes = r->bytes;
    sl->stream = st;
    if (cudaMalloc(&sl->d_mu, sl->vol * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&sl->d_x, sl->vol * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&sl->d_y, sl->proj * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&sl->d_s, 16) != cudaSuccess || cudaEventCreateWithFlags(&sl->done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        destroy_slot(sl);
        return SPECT_ENOMEM;
    }
    if (cudaMemcpyAsync(sl->d_mu, r->h_mu, sl->vol * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        destroy_slot(sl);
        return SPECT_ECUDA;
    }
    spect_geom g = sl->geom;
    g.angles_rad = sl->angles.empty() ? nullptr : sl->angles.data();
    g.det_offsets = sl->offsets.empty() ? nullptr : sl->offsets.data();
    g.det_shifts = sl->shifts.empty() ? nullptr : sl->shifts.data();
    g.fov_mask = sl->fov.empty() ? nullptr : sl->fov.data();
    int rc = spect_plan_create(&g, (g.flags & SPECT_FLAG_ATTEN) ? sl->d_mu : nullptr, st, &sl->plan);
    if (rc) {
        destroy_slot(sl);
        return rc;
    }
    sl->fresh = true;
    // capture one OSEM iteration (subsets 0..M-1), reading s from d_s
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const int orc = spect_osem_run_dev(sl->plan, sl->d_y, sl->d_s, sl->d_x, 0, g.n_subsets, nullptr, st);
        const cudaError_t ee = cudaStreamEndCapture(st, &graph);
        if (orc != SPECT_OK || ee != cudaSuccess || !graph || cudaGraphInstantiate(&sl->iter, graph, 0) != cudaSuccess)
            sl->iter = nullptr;  // replay the launches directly instead
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
    }
    (void)sv;
    *out = sl;
    return SPECT_OK;
}

// Queue request r on its slot: inputs, attenuation and sensitivities (unless
// the slot was just built from r), x = 1, n_iters iterations, read-back.
int start_request(spect_server* sv, Request* r, Slot* sl)
{
    cudaStream_t st = sl->stream;
    if (!sl->fresh) {
        if (cudaMemcpyAsync(sl->d_mu, r->h_mu, sl->vol * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return SPECT_ECUDA;
        const int rc = spect_plan_set_mu(sl->plan, (sl->geom.flags & SPECT_FLAG_ATTEN) ? sl->d_mu : nullptr, st);
        if (rc) return rc;
    }
    sl->fresh = false;
    if (cudaMemcpyAsync(sl->d_y, r->h_y, sl->proj * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return SPECT_ECUDA;
    if (spect::launch_fill(sl->d_s, 1, r->s, st) != cudaSuccess) return SPECT_ECUDA;
    if (spect::launch_fill(sl->d_x, sl->vol, 1.f, st) != cudaSuccess) return SPECT_ECUDA;
    for (int it = 0; it < r->n_iters; ++it) {
        if (sl->iter) {
            if (cudaGraphLaunch(sl->iter, st) != cudaSuccess) return SPECT_ECUDA;
        } else {
            const int rc = spect_osem_run_dev(sl->plan, sl->d_y, sl->d_s, sl->d_x, 0, sl->geom.n_subsets, nullptr, st);
            if (rc) return rc;
        }
    }
    if (cudaMemcpyAsync(r->h_x, sl->d_x, sl->vol * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SPECT_ECUDA;
    if (cudaEventRecord(sl->done, st) != cudaSuccess) return SPECT_ECUDA;
    // the pinned mu copy is no longer needed once the stream has consumed it;
    // it is returned when the request finishes (the stream is then past it)
    (void)sv;
    return SPECT_OK;
}

void finish(spect_server* sv, Request* r, int status, int state)
{
    // caller holds the lock
    r->status = status;
    r->state = state;
    r->t_done = now_ms();
    sv->pinned.give(r->h_mu);
    r->h_mu = nullptr;
    r->h_y = nullptr;  // the same pinned buffer now holds the image (h_x)
    if (state == SPECT_REQ_DONE) {
        sv->stats.completed += 1;
        sv->latencies.push_back(r->t_done - r->t_submit);
        sv->t_last_done = r->t_done;
    } else if (state == SPECT_REQ_FAILED) {
        sv->stats.failed += 1;
    }
    sv->cv_done.notify_all();
}

void scheduler(spect_server* sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->m);
    while (true) {
        // admit: FIFO, letting requests that can start now pass one that cannot
        for (auto it = sv->queue.begin(); it != sv->queue.end() && (int)sv->active.size() < sv->cfg.max_slots;) {
            Request* r = *it;
            if (r->cancel) {
                it = sv->queue.erase(it);
                r->state = SPECT_REQ_CANCELLED;
                r->status = SPECT_ECANCELLED;
                sv->pinned.give(r->h_mu);
                sv->pinned.give(r->h_y);
                r->h_mu = r->h_y = r->h_x = nullptr;
                sv->stats.cancelled += 1;
                sv->cv_done.notify_all();
                continue;
            }
            Slot* sl = nullptr;
            for (Slot* c : sv->slots)
                if (!c->busy && same_geometry(*c, *r)) {
                    sl = c;
                    break;
                }
            if (!sl) {
                // release idle slots of other geometries until a new one fits
                for (size_t k = 0; k < sv->slots.size() && sv->in_use + r->bytes > sv->cfg.hbm_budget_bytes;) {
                    Slot* c = sv->slots[k];
                    if (c->busy) {
                        ++k;
                        continue;
                    }
                    sv->slots.erase(sv->slots.begin() + k);
                    sv->in_use -= c->bytes;
                    destroy_slot(c);
                }
                if (sv->in_use + r->bytes > sv->cfg.hbm_budget_bytes) {
                    ++it;
                    continue;
                }
                sv->in_use += r->bytes;
                const cudaStream_t st = sv->streams[sv->next_stream++ % sv->streams.size()];
                lk.unlock();
                const int rc = create_slot(sv, r, st, &sl);
                lk.lock();
                if (rc) {
                    sv->in_use -= r->bytes;
                    it = sv->queue.erase(std::find(sv->queue.begin(), sv->queue.end(), r));
                    finish(sv, r, rc, SPECT_REQ_FAILED);
                    it = sv->queue.begin();
                    continue;
                }
                sv->slots.push_back(sl);
                sv->stats.slots_created += 1;
                if (sl->iter) sv->stats.graph_slots += 1;
                sv->stats.peak_bytes = std::max<uint64_t>(sv->stats.peak_bytes, sv->in_use);
            }
            sl->busy = true;
            sl->req = r;
            r->slot = sl;
            sv->queue.erase(std::find(sv->queue.begin(), sv->queue.end(), r));
            r->state = SPECT_REQ_RUNNING;
            r->t_admit = now_ms();
            sv->active.push_back(r);
            sv->stats.peak_active = std::max<uint64_t>(sv->stats.peak_active, sv->active.size());
            lk.unlock();
            const int rc = start_request(sv, r, sl);
            lk.lock();
            if (rc) {
                sv->active.erase(std::find(sv->active.begin(), sv->active.end(), r));
                cudaStreamSynchronize(sl->stream);
                sl->busy = false;
                sl->req = nullptr;
                finish(sv, r, rc, SPECT_REQ_FAILED);
            } else {
                sv->stats.admitted += 1;
            }
            it = sv->queue.begin();  // slots and budget changed: rescan from the head
        }
        // retire finished requests
        bool retired = false;
        for (size_t k = 0; k < sv->active.size();) {
            Request* r = sv->active[k];
            Slot* sl = r->slot;
            const cudaError_t q = cudaEventQuery(sl->done);
            if (q == cudaErrorNotReady) {
                ++k;
                continue;
            }
            sv->active.erase(sv->active.begin() + k);
            int status = q == cudaSuccess ? SPECT_OK : SPECT_ECUDA;
            if (status == SPECT_OK && spect_plan_check(sl->plan) != SPECT_OK) status = SPECT_ETIMEDOUT;
            cudaGetLastError();
            sl->busy = false;
            sl->req = nullptr;
            r->slot = nullptr;
            finish(sv, r, status, status == SPECT_OK ? SPECT_REQ_DONE : SPECT_REQ_FAILED);
            retired = true;
        }
        if (sv->stop && sv->queue.empty() && sv->active.empty()) break;
        if (retired) continue;
        if (sv->active.empty())
            sv->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        else
            sv->cv_work.wait_for(lk, std::chrono::microseconds(50));
    }
}

int sfail(int status, const char* msg)
{
    spect_internal_set_error(msg);
    return status;
}

}  // namespace

extern "C" {

int spect_serve_create(const spect_serve_cfg* cfg, spect_server** out)
{
    if (!out) return sfail(SPECT_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg) return sfail(SPECT_EINVAL, "cfg is NULL");
    if (cfg->max_slots < 1 || cfg->max_slots > 256) return sfail(SPECT_EINVAL, "max_slots must be in [1, 256]");
    if (cfg->n_streams < 1 || cfg->n_streams > 64) return sfail(SPECT_EINVAL, "n_streams must be in [1, 64]");
    if (cfg->hbm_budget_bytes < (1u << 20)) return sfail(SPECT_EINVAL, "hbm_budget_bytes below 1 MiB");
    if (cfg->wait_timeout_ms < 1) return sfail(SPECT_EINVAL, "wait_timeout_ms must be >= 1");
    spect_server* sv = new (std::nothrow) spect_server();
    if (!sv) return sfail(SPECT_ENOMEM, "host allocation failed");
    sv->cfg = *cfg;
    if (cudaGetDevice(&sv->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sv->num_sms, cudaDevAttrMultiProcessorCount, sv->device) != cudaSuccess) {
        cudaGetLastError();
        delete sv;
        return sfail(SPECT_ECUDA, "no CUDA device");
    }
    for (int k = 0; k < cfg->n_streams; ++k) {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (cudaStream_t t : sv->streams) cudaStreamDestroy(t);
            delete sv;
            return sfail(SPECT_ECUDA, "cudaStreamCreate failed");
        }
        sv->streams.push_back(s);
    }
    sv->worker = std::thread(scheduler, sv);
    *out = sv;
    return SPECT_OK;
}

int spect_serve_submit(spect_server* sv, const spect_request* req, uint64_t* id)
{
    if (!sv || !req || !id) return sfail(SPECT_EINVAL, "server, request and id must not be NULL");
    const spect_geom& g = req->geom;
    if (!req->y_host || ((g.flags & SPECT_FLAG_ATTEN) && !req->mu_host))
        return sfail(SPECT_EINVAL, "request needs y (and mu with attenuation)");
    if (req->n_iters < 1 || g.nx < 2 || g.nx != g.ny || g.nz < 4 || g.n_angles < 1 || g.n_subsets < 1 ||
        g.n_subsets > g.n_angles)
        return sfail(SPECT_EINVAL, "invalid request geometry or iteration count");
    if (!(req->s >= 0.f)) return sfail(SPECT_EINVAL, "s must be >= 0");
    auto* r = new (std::nothrow) Request();
    if (!r) return sfail(SPECT_ENOMEM, "host allocation failed");
    r->geom = g;
    r->geom.angles_rad = nullptr;
    r->geom.det_offsets = nullptr;
    r->geom.det_shifts = nullptr;
    r->geom.fov_mask = nullptr;
    if (g.angles_rad) r->angles.assign(g.angles_rad, g.angles_rad + g.n_angles);
    if (g.det_offsets) r->offsets.assign(g.det_offsets, g.det_offsets + g.n_angles);
    if (g.det_shifts) r->shifts.assign(g.det_shifts, g.det_shifts + g.n_angles);
    if (g.fov_mask) r->fov.assign(g.fov_mask, g.fov_mask + (size_t)g.n_angles * g.ny * g.nz);
    r->s = req->s;
    r->n_iters = req->n_iters;
    r->tag = req->tag;
    r->vol = (size_t)g.nx * g.ny * g.nz;
    r->proj = (size_t)g.n_angles * g.ny * g.nz;
    r->bytes = request_bytes(g, sv->num_sms);
    if (r->bytes > sv->cfg.hbm_budget_bytes) {
        delete r;
        std::lock_guard<std::mutex> lk(sv->m);
        sv->stats.rejected += 1;
        return sfail(SPECT_EBUDGET, "request needs more device memory than the whole budget");
    }
    r->h_mu = sv->pinned.take(r->vol);
    r->h_y = sv->pinned.take(std::max(r->proj, r->vol));
    r->h_x = r->h_y;  // the counts' pinned buffer receives the image at the end
    if (!r->h_mu || !r->h_y) {
        sv->pinned.give(r->h_mu);
        sv->pinned.give(r->h_y);
        delete r;
        return sfail(SPECT_ENOMEM, "pinned host allocation failed");
    }
    if (req->mu_host) std::memcpy(r->h_mu, req->mu_host, r->vol * sizeof(float));
    else std::memset(r->h_mu, 0, r->vol * sizeof(float));
    std::memcpy(r->h_y, req->y_host, r->proj * sizeof(float));
    {
        std::lock_guard<std::mutex> lk(sv->m);
        if (sv->stop) {
            sv->pinned.give(r->h_mu);
            sv->pinned.give(r->h_y);
            delete r;
            return sfail(SPECT_ESTATE, "server is shutting down");
        }
        r->id = sv->next_id++;
        r->t_submit = now_ms();
        if (sv->t_first_submit < 0) sv->t_first_submit = r->t_submit;
        sv->all[r->id] = r;
        sv->queue.push_back(r);
        sv->stats.submitted += 1;
        *id = r->id;
    }
    sv->cv_work.notify_one();
    return SPECT_OK;
}

int spect_serve_poll(spect_server* sv, uint64_t id, int* state)
{
    if (!sv || !state) return sfail(SPECT_EINVAL, "server and state must not be NULL");
    std::lock_guard<std::mutex> lk(sv->m);
    auto it = sv->all.find(id);
    if (it == sv->all.end()) return sfail(SPECT_ENOTFOUND, "unknown request id");
    *state = it->second->state;
    return SPECT_OK;
}

int spect_serve_wait(spect_server* sv, uint64_t id, int timeout_ms, float* x_host, double* latency_ms)
{
    if (!sv) return sfail(SPECT_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(sv->m);
    auto it = sv->all.find(id);
    if (it == sv->all.end()) return sfail(SPECT_ENOTFOUND, "unknown request id");
    Request* r = it->second;
    const int limit = timeout_ms > 0 ? timeout_ms : sv->cfg.wait_timeout_ms;
    const bool ended = sv->cv_done.wait_for(lk, std::chrono::milliseconds(limit), [r] {
        return r->state == SPECT_REQ_DONE || r->state == SPECT_REQ_FAILED || r->state == SPECT_REQ_CANCELLED;
    });
    if (!ended) return sfail(SPECT_ETIMEDOUT, "request did not finish within the timeout");
    const int status = r->status;
    if (status == SPECT_OK && x_host) std::memcpy(x_host, r->h_x, r->vol * sizeof(float));
    if (latency_ms) *latency_ms = r->t_done - r->t_submit;
    sv->pinned.give(r->h_x);
    sv->all.erase(it);
    delete r;
    if (status != SPECT_OK)
        return sfail(status, status == SPECT_ECANCELLED ? "request was cancelled" : "request failed on the device");
    return SPECT_OK;
}

int spect_serve_cancel(spect_server* sv, uint64_t id)
{
    if (!sv) return sfail(SPECT_EINVAL, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(sv->m);
        auto it = sv->all.find(id);
        if (it == sv->all.end()) return sfail(SPECT_ENOTFOUND, "unknown request id");
        if (it->second->state != SPECT_REQ_QUEUED)
            return sfail(SPECT_ESTATE, "only queued requests can be cancelled");
        it->second->cancel = true;
    }
    sv->cv_work.notify_one();
    return SPECT_OK;
}

int spect_serve_stats_get(spect_server* sv, spect_serve_stats* out)
{
    if (!sv || !out) return sfail(SPECT_EINVAL, "server and out must not be NULL");
    std::lock_guard<std::mutex> lk(sv->m);
    *out = sv->stats;
    out->queued = sv->queue.size();
    out->active = sv->active.size();
    out->bytes_in_use = sv->in_use;
    std::vector<double> lat = sv->latencies;
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double q) {
        if (lat.empty()) return 0.0;
        const size_t k = std::min(lat.size() - 1, (size_t)(q * (double)(lat.size() - 1) + 0.5));
        return lat[k];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = lat.empty() ? 0.0 : lat.back();
    const double span = sv->t_last_done - sv->t_first_submit;
    out->recon_per_s = (span > 0 && !lat.empty()) ? 1e3 * (double)lat.size() / span : 0.0;
    return SPECT_OK;
}

int spect_serve_destroy(spect_server* sv)
{
    if (!sv) return SPECT_OK;
    {
        std::lock_guard<std::mutex> lk(sv->m);
        sv->stop = true;
        for (Request* r : sv->queue) r->cancel = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (auto& kv : sv->all) {
        Request* r = kv.second;
        sv->pinned.give(r->h_mu);
        sv->pinned.give(r->h_x);  // also the counts buffer (same allocation)
        delete r;
    }
    for (Slot* sl : sv->slots) destroy_slot(sl);
    sv->slots.clear();
    for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
    delete sv;
    return SPECT_OK;
}

}  // extern "C"
