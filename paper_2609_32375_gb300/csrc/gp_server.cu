// gp_server.cu -- the request server of include/gpphot.h: continuous
// batching of frames from host memory under a device-memory budget.
//
// The paper runs several worker processes on one GPU and bounds how many
// frames they can hold at once by usable device memory over one frame's peak
// working set (Section 6.4).  Here one process owns the GPU and applies that
// bound per request: the device budget is one allocation made at start-up,
// carved first-fit into per-unit regions (pixels, segmentation maps,
// workspace, results), so admission never exceeds it and nothing is
// allocated while serving.
//
//  submit   validates the request, computes its footprint, queues it.
//  worker   one thread; admits queued requests in arrival order when a slot
//           (a stream with its own pinned argument staging) is free and the
//           unit's footprint fits both pools.  Consecutive small frames at
//           the head of the queue form one unit, run by the batched pipeline
//           (every stage one launch over the unit's frames).  A unit is:
//           host-to-device copies, the pipeline, one device-to-host copy of
//           the unit's result blocks, then a host callback that hands the
//           unit back to the worker.  Units on different slots overlap.
//  wait     blocks (bounded) until the request's result is ready.
//  release  returns the result's pinned host memory to the pool.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gp_pipeline.h"

using namespace gp;

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

size_t round_up(size_t n, size_t a) { return (n + a - 1) / a * a; }

gp_status srv_fail(gp_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    record_error(buf);
    return s;
}

// first-fit allocator over [0, size) with coalescing on free
class Pool {
public:
    void init(size_t size)
    {
        size_ = size;
        free_.clear();
        free_[0] = size;
        used_ = peak_ = 0;
    }
    bool alloc(size_t n, size_t* off)
    {
        n = round_up(n ? n : 1, ALIGN);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n, at = it->first + n;
            free_.erase(it);
            if (rest) free_[at] = rest;
            used_ += n;
            peak_ = std::max(peak_, used_);
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = round_up(n ? n : 1, ALIGN);
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }
    size_t peak() const { return peak_; }
    void reset_peak() { peak_ = used_; }

private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, used_ = 0, peak_ = 0;
};

// A frame's result block (identical layout on the device and in pinned host
// memory, so one copy moves it): header (status, segment count), catalog
// columns of `capacity` rows, aperture arrays of capacity*nr, meshes.
struct ResultLayout {
    size_t label, npix, flux_iso, x, y, x2, y2, xy, xmin, xmax, ymin, ymax, peak, xpeak, ypeak, flags;
    size_t apflux, apferr, apflags, bkg, rms, total;
};

ResultLayout result_layout(int cap, int nr, int nbox)
{
    ResultLayout L;
    size_t off = ALIGN;   // header
    auto col = [&](size_t bytes) {
        const size_t o = off;
        off = round_up(off + bytes, ALIGN);
        return o;
    };
    const size_t c = (size_t)cap;
    L.label = col(4 * c); L.npix = col(4 * c); L.flux_iso = col(8 * c);
    L.x = col(8 * c); L.y = col(8 * c); L.x2 = col(8 * c); L.y2 = col(8 * c); L.xy = col(8 * c);
    L.xmin = col(4 * c); L.xmax = col(4 * c); L.ymin = col(4 * c); L.ymax = col(4 * c);
    L.peak = col(4 * c); L.xpeak = col(4 * c); L.ypeak = col(4 * c); L.flags = col(4 * c);
    L.apflux = col(8 * c * nr); L.apferr = col(8 * c * nr); L.apflags = col(4 * c * nr);
    L.bkg = col(4 * (size_t)nbox); L.rms = col(4 * (size_t)nbox);
    L.total = off;
    return L;
}

template <class T>
T* at(char* base, size_t off) { return reinterpret_cast<T*>(base + off); }

struct Unit;

struct Req {
    uint64_t id;
    gp_request r;
    int W, H, Mx, My;
    int64_t npix;
    size_t esize;
    Clock::time_point t_submit, t_admit;
    bool done = false;
    int32_t n_host = 0;
    gp_result res;
    std::string msg;
    Unit* unit = nullptr;
};

struct Unit {
    int slot;
    std::vector<Req*> frames;
    size_t dev_off, dev_bytes, host_off, host_bytes;
    size_t rb;             // result block bytes (uniform within the unit)
    size_t seg_host_off;   // first host segmentation map (after the result blocks)
    int refs = 0;          // results not yet released
};

struct Slot {
    cudaStream_t st = nullptr;
    SideStream side{nullptr, nullptr, nullptr};   // the crowded tiles' labelling beside st
    ArgStage stage;
    Unit* unit = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};   // unit start, inputs in, pipeline done, results out
};

}  // namespace

struct gp_server {
    gp_server_config cfg;
    Params P;
    char* dpool = nullptr;
    char* hpool = nullptr;
    Pool dp, hp;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> queue;
    std::unordered_map<uint64_t, Req*> reqs;
    std::vector<Unit*> finished;      // units whose stream reached their callback
    uint64_t next_id = 1;
    bool stop = false, kick = false;
    int inflight = 0;
    std::thread worker;
    // counters
    int64_t submitted = 0, completed = 0, failed = 0, units = 0, batched_frames = 0;
    double mpix = 0;
    int peak_inflight = 0;
    std::vector<double> lat;
    bool any_submit = false;
    Clock::time_point t_first, t_last;

    size_t unit_device_bytes(const std::vector<Req*>& fr, size_t* rb_out) const;
    size_t unit_host_bytes(const std::vector<Req*>& fr, size_t rb) const;
    void admit(std::unique_lock<std::mutex>& lk);
    gp_status launch(Unit* u);
    void finish(Unit* u);
    void fail_unit(Unit* u, gp_status s, const std::string& msg);
    void run();
};

namespace {

void CUDART_CB on_unit_done(void* arg)
{
    auto* pr = static_cast<std::pair<gp_server*, Unit*>*>(arg);
    gp_server* s = pr->first;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->finished.push_back(pr->second);
        s->kick = true;
    }
    s->cv_work.notify_one();
    delete pr;
}

}  // namespace

size_t gp_server::unit_device_bytes(const std::vector<Req*>& fr, size_t* rb_out) const
{
    const int n = (int)fr.size();
    size_t rb = 0;
    std::vector<int> W(n), H(n), C(n);
    for (int f = 0; f < n; ++f) {
        rb = std::max(rb, result_layout(fr[f]->r.capacity, P.nr, fr[f]->Mx * fr[f]->My).total);
        W[f] = fr[f]->W; H[f] = fr[f]->H; C[f] = fr[f]->r.capacity;
    }
    size_t b = n * rb;
    for (int f = 0; f < n; ++f) {
        b = round_up(b, ALIGN) + (size_t)fr[f]->npix * fr[f]->esize;                       // pixels
        if (fr[f]->r.image.mask) b = round_up(b, ALIGN) + (size_t)fr[f]->npix;               // mask
        b = round_up(b, ALIGN) + (size_t)fr[f]->npix * 4;                                   // segmentation map
    }
    b = round_up(b, ALIGN) + extract_workspace_bytes(n, W.data(), H.data(), C.data(), P.bp.mesh, P.net != nullptr) +
        (64 << 10);
    if (rb_out) *rb_out = rb;
    return b;
}

size_t gp_server::unit_host_bytes(const std::vector<Req*>& fr, size_t rb) const
{
    size_t b = fr.size() * rb;
    for (Req* q : fr)
        if (q->r.want_segmap) b = round_up(b, ALIGN) + (size_t)q->npix * 4;
    return b;
}

void gp_server::admit(std::unique_lock<std::mutex>& lk)
{
    while (!queue.empty() && !stop) {
        int slot = -1;
        for (int i = 0; i < (int)slots.size(); ++i)
            if (!slots[i].unit) { slot = i; break; }
        if (slot < 0) return;
        Req* head = queue.front();
        std::vector<Req*> pick{head};
        if (head->npix <= cfg.batch_pixels && cfg.max_batch > 1) {
            for (size_t i = 1; i < queue.size() && (int)pick.size() < cfg.max_batch; ++i) {
                Req* q = queue[i];
                if (q->npix > cfg.batch_pixels || q->r.image.dtype != head->r.image.dtype) break;
                if (P.net && (q->Mx != head->Mx || q->My != head->My)) break;
                pick.push_back(q);
            }
        }
        size_t doff = 0, hoff = 0, dbytes = 0, hbytes = 0, rb = 0;
        for (;;) {
            dbytes = unit_device_bytes(pick, &rb);
            hbytes = unit_host_bytes(pick, rb);
            if (dp.alloc(dbytes, &doff)) {
                if (hp.alloc(hbytes, &hoff)) break;
                dp.release(doff, dbytes);
            }
            if (pick.size() == 1) return;     // the head waits for memory; so does everything behind it
            pick.pop_back();
        }
        const Clock::time_point now = Clock::now();
        Unit* u = new Unit;
        u->slot = slot;
        u->frames = pick;
        u->dev_off = doff; u->dev_bytes = dbytes;
        u->host_off = hoff; u->host_bytes = hbytes;
        u->rb = rb;
        u->seg_host_off = pick.size() * rb;
        for (Req* q : pick) {
            q->t_admit = now;
            q->unit = u;
            queue.pop_front();
        }
        slots[slot].unit = u;
        ++inflight;
        peak_inflight = std::max(peak_inflight, inflight);
        ++units;
        if (pick.size() > 1) batched_frames += (int64_t)pick.size();
        lk.unlock();
        const gp_status s = launch(u);
        lk.lock();
        if (s != GP_OK) fail_unit(u, s, gp_last_error());
    }
}

gp_status gp_server::launch(Unit* u)
{
    Slot& sl = slots[u->slot];
    cudaStream_t st = sl.st;
    const int n = (int)u->frames.size();
    char* dbase = dpool + u->dev_off;
    char* hbase = hpool + u->host_off;
    std::vector<ResultLayout> L(n);
    std::vector<FrameIO> F(n);
    size_t off = n * u->rb;
    for (int f = 0; f < n; ++f) {
        Req* q = u->frames[f];
        L[f] = result_layout(q->r.capacity, P.nr, q->Mx * q->My);
    }
    std::vector<char*> dimg(n), dmask(n, nullptr), dseg(n);
    for (int f = 0; f < n; ++f) {
        Req* q = u->frames[f];
        off = round_up(off, ALIGN);
        dimg[f] = dbase + off;
        off += (size_t)q->npix * q->esize;
        if (q->r.image.mask) {
            off = round_up(off, ALIGN);
            dmask[f] = dbase + off;
            off += (size_t)q->npix;
        }
        off = round_up(off, ALIGN);
        dseg[f] = dbase + off;
        off += (size_t)q->npix * 4;
    }
    off = round_up(off, ALIGN);
    const size_t ws_bytes = u->dev_bytes - off;
    char* dws = dbase + off;

    // inputs
    cudaEventRecord(sl.ev[0], st);
    for (int f = 0; f < n; ++f) {
        Req* q = u->frames[f];
        const size_t row = (size_t)q->W * q->esize;
        cudaError_t e = cudaMemcpy2DAsync(dimg[f], row, q->r.image.data, (size_t)q->r.image.pitch * q->esize, row,
                                          (size_t)q->H, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && dmask[f])
            e = cudaMemcpyAsync(dmask[f], q->r.image.mask, (size_t)q->npix, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return srv_fail(GP_ERR_CUDA, "input copy: %s", cudaGetErrorString(e));
    }
    // clear every frame's header (status word and count)
    cudaError_t e = cudaMemset2DAsync(dbase, u->rb, 0, ALIGN, (size_t)n, st);
    if (e != cudaSuccess) return srv_fail(GP_ERR_CUDA, "header clear: %s", cudaGetErrorString(e));
    for (int f = 0; f < n; ++f) {
        Req* q = u->frames[f];
        char* r = dbase + f * u->rb;
        FrameIO& x = F[f];
        memset(&x, 0, sizeof x);
        x.img = q->r.image;
        x.img.data = dimg[f];
        x.img.pitch = q->W;
        x.img.mask = reinterpret_cast<const uint8_t*>(dmask[f]);
        x.bkg.bkg_mesh = at<float>(r, L[f].bkg);
        x.bkg.rms_mesh = at<float>(r, L[f].rms);
        x.segmap = reinterpret_cast<uint32_t*>(dseg[f]);
        gp_catalog& c = x.cat;
        c.capacity = q->r.capacity;
        c.n = at<int32_t>(r, 4);
        c.label = at<uint32_t>(r, L[f].label); c.npix = at<int32_t>(r, L[f].npix);
        c.flux_iso = at<double>(r, L[f].flux_iso);
        c.x = at<double>(r, L[f].x); c.y = at<double>(r, L[f].y);
        c.x2 = at<double>(r, L[f].x2); c.y2 = at<double>(r, L[f].y2); c.xy = at<double>(r, L[f].xy);
        c.xmin = at<int32_t>(r, L[f].xmin); c.xmax = at<int32_t>(r, L[f].xmax);
        c.ymin = at<int32_t>(r, L[f].ymin); c.ymax = at<int32_t>(r, L[f].ymax);
        c.peak = at<float>(r, L[f].peak);
        c.xpeak = at<int32_t>(r, L[f].xpeak); c.ypeak = at<int32_t>(r, L[f].ypeak);
        c.flags = at<uint32_t>(r, L[f].flags);
        x.apflux = at<double>(r, L[f].apflux);
        x.apferr = at<double>(r, L[f].apferr);
        x.apflags = at<uint32_t>(r, L[f].apflags);
        x.status = at<int>(r, 0);
    }
    cudaEventRecord(sl.ev[1], st);
    Exec ex;
    ex.cv = Carver{dws, ws_bytes};
    ex.st = st;
    ex.side = &sl.side;
    ex.stage = &sl.stage;
    gp_status s = run_extract(ex, n, F.data(), P);
    if (s == GP_ERR_OOM)
        return srv_fail(GP_ERR_INTERNAL, "unit workspace of %zu bytes short of the %zu carved", ws_bytes, ex.cv.off);
    if (s != GP_OK) return s;
    // results back: the unit's result blocks in one copy, then the wanted maps
    cudaEventRecord(sl.ev[2], st);
    e = cudaMemcpyAsync(hbase, dbase, n * u->rb, cudaMemcpyDeviceToHost, st);
    size_t hoff = u->seg_host_off;
    for (int f = 0; f < n && e == cudaSuccess; ++f) {
        Req* q = u->frames[f];
        if (!q->r.want_segmap) continue;
        hoff = round_up(hoff, ALIGN);
        e = cudaMemcpyAsync(hbase + hoff, dseg[f], (size_t)q->npix * 4, cudaMemcpyDeviceToHost, st);
        hoff += (size_t)q->npix * 4;
    }
    if (e != cudaSuccess) return srv_fail(GP_ERR_CUDA, "result copy: %s", cudaGetErrorString(e));
    cudaEventRecord(sl.ev[3], st);
    auto* arg = new std::pair<gp_server*, Unit*>(this, u);
    e = cudaLaunchHostFunc(st, on_unit_done, arg);
    if (e != cudaSuccess) {
        delete arg;
        return srv_fail(GP_ERR_CUDA, "completion callback: %s", cudaGetErrorString(e));
    }
    return GP_OK;
}

// with mu held: results of a unit whose stream completed
void gp_server::finish(Unit* u)
{
    const Clock::time_point now = Clock::now();
    // a failed copy or kernel makes the stream's error visible here
    const cudaError_t e = cudaStreamQuery(slots[u->slot].st);
    char* hbase = hpool + u->host_off;
    const int n = (int)u->frames.size();
    size_t hoff = u->seg_host_off;
    float t_in = 0.f, t_run = 0.f, t_out = 0.f;
    const cudaEvent_t* ev = slots[u->slot].ev;
    if (cudaEventElapsedTime(&t_in, ev[0], ev[1]) != cudaSuccess || cudaEventElapsedTime(&t_run, ev[1], ev[2]) !=
        cudaSuccess || cudaEventElapsedTime(&t_out, ev[2], ev[3]) != cudaSuccess)
        t_in = t_run = t_out = -1.f;
    for (int f = 0; f < n; ++f) {
        Req* q = u->frames[f];
        char* r = hbase + f * u->rb;
        const ResultLayout L = result_layout(q->r.capacity, P.nr, q->Mx * q->My);
        gp_result& res = q->res;
        memset(&res, 0, sizeof res);
        const int32_t* hdr = at<int32_t>(r, 0);
        res.status = (e == cudaSuccess || e == cudaErrorNotReady) ? hdr[0] : GP_ERR_CUDA;
        res.n = hdr[1];
        q->n_host = hdr[1];
        gp_catalog& c = res.cat;
        c.capacity = q->r.capacity;
        c.n = &q->n_host;
        c.label = at<uint32_t>(r, L.label); c.npix = at<int32_t>(r, L.npix);
        c.flux_iso = at<double>(r, L.flux_iso);
        c.x = at<double>(r, L.x); c.y = at<double>(r, L.y);
        c.x2 = at<double>(r, L.x2); c.y2 = at<double>(r, L.y2); c.xy = at<double>(r, L.xy);
        c.xmin = at<int32_t>(r, L.xmin); c.xmax = at<int32_t>(r, L.xmax);
        c.ymin = at<int32_t>(r, L.ymin); c.ymax = at<int32_t>(r, L.ymax);
        c.peak = at<float>(r, L.peak);
        c.xpeak = at<int32_t>(r, L.xpeak); c.ypeak = at<int32_t>(r, L.ypeak);
        c.flags = at<uint32_t>(r, L.flags);
        res.flux = at<double>(r, L.apflux);
        res.fluxerr = at<double>(r, L.apferr);
        res.apflags = at<uint32_t>(r, L.apflags);
        res.bkg_mesh = at<float>(r, L.bkg);
        res.rms_mesh = at<float>(r, L.rms);
        res.mesh = P.bp.mesh; res.mx = q->Mx; res.my = q->My;
        if (q->r.want_segmap) {
            hoff = round_up(hoff, ALIGN);
            res.segmap = at<uint32_t>(hbase, hoff);
            hoff += (size_t)q->npix * 4;
        }
        res.batch = n;
        res.h2d_ms = t_in;
        res.run_ms = t_run;
        res.d2h_ms = t_out;
        res.latency_ms = ms_between(q->t_submit, now);
        res.queue_ms = ms_between(q->t_submit, q->t_admit);
        if (res.status == GP_ERR_CAPACITY) q->msg = "more segments than catalog rows (see n)";
        else if (res.status == GP_ERR_TIMEOUT) q->msg = "a bounded device-side walk gave up";
        else if (res.status == GP_ERR_INTERNAL) q->msg = "an internal device table overflowed";
        else if (res.status == GP_ERR_CUDA) q->msg = std::string("CUDA error: ") + cudaGetErrorString(e);
        q->done = true;
        if (res.status == GP_OK) {
            ++completed;
            mpix += (double)q->npix * 1e-6;
            lat.push_back(res.latency_ms);
        } else {
            ++failed;
        }
    }
    t_last = now;
    u->refs = n;
    dp.release(u->dev_off, u->dev_bytes);
    slots[u->slot].unit = nullptr;
    --inflight;
}

// with mu held: a unit that could not be launched (nothing of it in flight)
void gp_server::fail_unit(Unit* u, gp_status s, const std::string& msg)
{
    // work already enqueued on the stream must finish before its memory is reused
    cudaStreamSynchronize(slots[u->slot].st);
    for (Req* q : u->frames) {
        memset(&q->res, 0, sizeof q->res);
        q->res.status = s;
        q->res.batch = (int)u->frames.size();
        q->msg = msg;
        q->done = true;
        ++failed;
    }
    u->refs = (int)u->frames.size();
    dp.release(u->dev_off, u->dev_bytes);
    slots[u->slot].unit = nullptr;
    --inflight;
    cv_done.notify_all();
}

void gp_server::run()
{
    cudaSetDevice(cfg.device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        kick = false;
        bool any = false;
        while (!finished.empty()) {
            Unit* u = finished.back();
            finished.pop_back();
            finish(u);
            any = true;
        }
        if (any) cv_done.notify_all();
        if (stop) {
            // requests not yet admitted fail; work in flight finishes
            while (!queue.empty()) {
                Req* q = queue.front();
                queue.pop_front();
                memset(&q->res, 0, sizeof q->res);
                q->res.status = GP_ERR_INVALID_ARG;
                q->msg = "the server was shut down before this request was admitted";
                q->done = true;
                ++failed;
            }
            cv_done.notify_all();
            if (inflight == 0) break;
        } else {
            admit(lk);
        }
        if (kick) continue;
        cv_work.wait(lk, [&] { return kick; });
    }
}

extern "C" {

gp_status gp_server_create(const gp_server_config* cfg, gp_server** out)
{
    if (!out) return srv_fail(GP_ERR_INVALID_ARG, "null output pointer");
    *out = nullptr;
    if (!cfg) return srv_fail(GP_ERR_INVALID_ARG, "null configuration");
    if (cfg->slots < 1 || cfg->slots > 16) return srv_fail(GP_ERR_INVALID_ARG, "slots %d outside [1, 16]", cfg->slots);
    if (cfg->max_batch < 1 || cfg->max_batch > GP_MAX_BATCH)
        return srv_fail(GP_ERR_INVALID_ARG, "max_batch %d outside [1, %d]", cfg->max_batch, GP_MAX_BATCH);
    if (cfg->batch_pixels < 0) return srv_fail(GP_ERR_INVALID_ARG, "negative batch_pixels");
    if (cfg->hbm_budget < ((size_t)1 << 20) || cfg->host_budget < ((size_t)1 << 20))
        return srv_fail(GP_ERR_INVALID_ARG, "budgets must be at least 1 MiB");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return srv_fail(GP_ERR_CUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
    if (cfg->device < 0 || cfg->device >= ndev)
        return srv_fail(GP_ERR_INVALID_ARG, "device %d not present (%d devices)", cfg->device, ndev);
    gp_image probe{};
    probe.dtype = GP_U16;
    probe.width = probe.height = 1;
    gp_status s = validate_bkg_params(&probe, &cfg->bkg);
    if (s != GP_OK) return s;
    float taps[KMAX];
    if ((s = validate_det_params(&cfg->det, taps)) != GP_OK) return s;
    if ((s = validate_ap_params(&cfg->ap)) != GP_OK) return s;
    if (cfg->net && (s = validate_net(cfg->net)) != GP_OK) return s;
    e = cudaSetDevice(cfg->device);
    if (e != cudaSuccess) return srv_fail(GP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));

    gp_server* sv = new gp_server;
    sv->cfg = *cfg;
    Params& P = sv->P;
    memset(&P, 0, sizeof P);
    P.bp = cfg->bkg;
    for (int i = 0; i < cfg->det.kw * cfg->det.kh; ++i) P.taps[i] = taps[i];
    P.kw = cfg->det.kw; P.kh = cfg->det.kh;
    P.thresh = cfg->det.thresh;
    P.minarea = cfg->det.minarea;
    P.nr = cfg->ap.nr;
    for (int k = 0; k < cfg->ap.nr; ++k) P.radii[k] = cfg->ap.radii[k];
    P.gain = cfg->ap.gain;
    P.net = cfg->net;
    sv->cfg.det.kernel = nullptr;          // copied into P
    sv->cfg.ap.radii = nullptr;
    auto undo = [&](gp_status st, const char* what, cudaError_t err) {
        for (Slot& sl : sv->slots) {
            sl.stage.release();
            for (cudaEvent_t& x : sl.ev)
                if (x) cudaEventDestroy(x);
            if (sl.side.fork) cudaEventDestroy(sl.side.fork);
            if (sl.side.join) cudaEventDestroy(sl.side.join);
            if (sl.side.st) cudaStreamDestroy(sl.side.st);
            if (sl.st) cudaStreamDestroy(sl.st);
        }
        if (sv->dpool) cudaFree(sv->dpool);
        if (sv->hpool) cudaFreeHost(sv->hpool);
        delete sv;
        return srv_fail(st, "%s: %s", what, cudaGetErrorString(err));
    };
    e = cudaMalloc(reinterpret_cast<void**>(&sv->dpool), cfg->hbm_budget);
    if (e != cudaSuccess) return undo(GP_ERR_OOM, "device budget allocation", e);
    e = cudaHostAlloc(reinterpret_cast<void**>(&sv->hpool), cfg->host_budget, cudaHostAllocDefault);
    if (e != cudaSuccess) return undo(GP_ERR_OOM, "pinned host budget allocation", e);
    sv->dp.init(cfg->hbm_budget);
    sv->hp.init(cfg->host_budget);
    sv->slots.resize(cfg->slots);
    for (Slot& sl : sv->slots) {
        e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
        for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreate(&sl.ev[k]);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.side.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.side.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.side.join, cudaEventDisableTiming);
        if (e == cudaSuccess) e = sl.stage.init((size_t)512 << 10);
        if (e != cudaSuccess) return undo(GP_ERR_CUDA, "slot streams", e);
    }
    sv->worker = std::thread([sv] { sv->run(); });
    *out = sv;
    return GP_OK;
}

namespace {

// a validated request record (not yet queued), or null with the error set
Req* make_req(const gp_server* s, const gp_request* req, gp_status* st)
{
    *st = validate_image(&req->image);
    if (*st != GP_OK) return nullptr;
    if ((*st = validate_bkg_params(&req->image, &s->P.bp)) != GP_OK) return nullptr;
    if (req->capacity < 1) {
        *st = srv_fail(GP_ERR_INVALID_ARG, "capacity %d < 1", req->capacity);
        return nullptr;
    }
    Req* q = new Req;
    q->r = *req;
    q->W = req->image.width;
    q->H = req->image.height;
    q->npix = (int64_t)q->W * q->H;
    q->Mx = (q->W + s->P.bp.mesh - 1) / s->P.bp.mesh;
    q->My = (q->H + s->P.bp.mesh - 1) / s->P.bp.mesh;
    q->esize = req->image.dtype == GP_F32 ? 4 : 2;
    return q;
}

}  // namespace

gp_status gp_server_request_bytes(const gp_server* s, const gp_request* req, size_t* device_bytes, size_t* host_bytes)
{
    if (!s || !req || !device_bytes || !host_bytes) return srv_fail(GP_ERR_INVALID_ARG, "null argument");
    gp_status st;
    Req* q = make_req(s, req, &st);
    if (!q) return st;
    size_t rb = 0;
    const std::vector<Req*> one{q};
    *device_bytes = s->unit_device_bytes(one, &rb);
    *host_bytes = s->unit_host_bytes(one, rb);
    delete q;
    return GP_OK;
}

gp_status gp_server_submit(gp_server* s, const gp_request* req, uint64_t* ticket)
{
    if (!s || !req || !ticket) return srv_fail(GP_ERR_INVALID_ARG, "null server, request or ticket");
    gp_status st;
    Req* q = make_req(s, req, &st);
    if (!q) return st;
    size_t rb = 0;
    const std::vector<Req*> one{q};
    const size_t dbytes = s->unit_device_bytes(one, &rb), hbytes = s->unit_host_bytes(one, rb);
    if (dbytes > s->dp.size() || hbytes > s->hp.size()) {
        delete q;
        return srv_fail(GP_ERR_OOM, "request needs %zu device / %zu host bytes; budgets are %zu / %zu", dbytes, hbytes,
                        s->dp.size(), s->hp.size());
    }
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->stop) {
            delete q;
            return srv_fail(GP_ERR_INVALID_ARG, "server is shutting down");
        }
        q->id = s->next_id++;
        q->t_submit = Clock::now();
        if (!s->any_submit) {
            s->any_submit = true;
            s->t_first = q->t_submit;
        }
        s->reqs[q->id] = q;
        s->queue.push_back(q);
        ++s->submitted;
        s->kick = true;
        *ticket = q->id;
    }
    s->cv_work.notify_one();
    return GP_OK;
}

gp_status gp_server_wait(gp_server* s, uint64_t ticket, int32_t timeout_ms, gp_result* out)
{
    if (!s || !out) return srv_fail(GP_ERR_INVALID_ARG, "null server or result");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return srv_fail(GP_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    Req* q = it->second;
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, [&] { return q->done; });
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return q->done; })) {
        return srv_fail(GP_ERR_TIMEOUT, "request %llu not done after %d ms", (unsigned long long)ticket, timeout_ms);
    }
    *out = q->res;
    if (q->res.status != GP_OK) record_error(q->msg.c_str());
    return (gp_status)q->res.status;
}

gp_status gp_server_release(gp_server* s, uint64_t ticket)
{
    if (!s) return srv_fail(GP_ERR_INVALID_ARG, "null server");
    bool kick = false;
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return srv_fail(GP_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
        Req* q = it->second;
        if (!q->done) return srv_fail(GP_ERR_INVALID_ARG, "request %llu is not done", (unsigned long long)ticket);
        Unit* u = q->unit;
        s->reqs.erase(it);
        delete q;
        if (u && --u->refs == 0) {
            s->hp.release(u->host_off, u->host_bytes);
            delete u;
            s->kick = kick = true;        // host memory freed: admission may proceed
        }
    }
    if (kick) s->cv_work.notify_one();
    return GP_OK;
}

gp_status gp_server_stats(gp_server* s, gp_server_report* out, int32_t reset)
{
    if (!s || !out) return srv_fail(GP_ERR_INVALID_ARG, "null server or report");
    std::lock_guard<std::mutex> g(s->mu);
    memset(out, 0, sizeof *out);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->units = s->units;
    out->batched_frames = s->batched_frames;
    out->mpix = s->mpix;
    out->wall_s = s->any_submit && s->completed ? ms_between(s->t_first, s->t_last) * 1e-3 : 0.0;
    if (!s->lat.empty()) {
        std::vector<double> v = s->lat;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            // nearest rank
            size_t k = (size_t)std::ceil(p * v.size());
            if (k < 1) k = 1;
            return v[std::min(k, v.size()) - 1];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_ms = sum / v.size();
        out->max_ms = v.back();
    }
    out->budget = s->dp.size();
    out->peak_bytes = s->dp.peak();
    out->peak_inflight = s->peak_inflight;
    if (reset) {
        s->submitted = s->completed = s->failed = s->units = s->batched_frames = 0;
        s->mpix = 0;
        s->lat.clear();
        s->any_submit = false;
        s->dp.reset_peak();
        s->peak_inflight = s->inflight;
    }
    return GP_OK;
}

void gp_server_destroy(gp_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        s->kick = true;
    }
    s->cv_work.notify_one();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->cfg.device);
    std::vector<Unit*> units;
    for (auto& kv : s->reqs) {
        Unit* u = kv.second->unit;
        if (u && std::find(units.begin(), units.end(), u) == units.end()) units.push_back(u);
        delete kv.second;
    }
    for (Unit* u : units) delete u;
    for (Slot& sl : s->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        if (sl.side.st) cudaStreamSynchronize(sl.side.st);
        sl.stage.release();
        for (cudaEvent_t& x : sl.ev)
            if (x) cudaEventDestroy(x);
        if (sl.side.fork) cudaEventDestroy(sl.side.fork);
        if (sl.side.join) cudaEventDestroy(sl.side.join);
        if (sl.side.st) cudaStreamDestroy(sl.side.st);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    cudaFree(s->dpool);
    cudaFreeHost(s->hpool);
    delete s;
}

}  // extern "C"
