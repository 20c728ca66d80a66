// Continuous-batching server of tactile steps (include/tacsl_serve.h): host runtime.
//
// Included at the end of tacsl.cu: it drives the batched kernels through the same
// internal functions as tacsl_batch_step (plan, pack, image and force launches).
//
// Threads: callers submit and wait under one mutex; ONE worker thread owns the CUDA
// work.  The worker loop:
//   1. retires finished batches (cudaEventQuery on each batch's completion event),
//      marking their requests done and returning their arena block; a batch still
//      running after batch_timeout_ms fails its requests with TACSL_ERR_TIMEOUT but keeps
//      its block until the GPU is done with it;
//   2. while a stream is free and requests wait, forms a batch of the oldest pending
//      requests of one kind whose memory fits in the largest free arena block (and
//      within max_pads), then - outside the lock - plans and packs it, copies every
//      request's inputs into the batch's arrays, renders the depth maps of a batch of
//      pose requests, launches the image and force kernels, copies every request's
//      outputs back to its host buffers and records an event, all on that stream;
//   3. sleeps until a request arrives or, while batches run, for a few microseconds.
// Each batch's arrays are one contiguous arena block: per request the pads, taxels
// and pixels are consecutive, so each request's data moves with one copy per array.
#pragma once

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <thread>

#include "tacsl_serve.h"

namespace tacsl {
namespace serve {

using Clock = std::chrono::steady_clock;

constexpr int64_t kGranule = 256;

int64_t round_up(int64_t n) { return (n + kGranule - 1) / kGranule * kGranule; }

// First-fit allocator of offsets in one device arena, neighbours coalesced on release.
class Arena {
  public:
    void init(int64_t size) {
        size_ = size;
        free_.clear();
        free_[0] = size;
        used_ = peak_ = 0;
    }
    int64_t largest_free() const {
        int64_t m = 0;
        for (const auto& f : free_) m = std::max(m, f.second);
        return m;
    }
    int64_t alloc(int64_t n) {
        n = round_up(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const int64_t off = it->first, rest = it->second - n;
            free_.erase(it);
            if (rest > 0) free_[off + n] = rest;
            used_ += n;
            peak_ = std::max(peak_, used_);
            return off;
        }
        return -1;
    }
    void release(int64_t off, int64_t n) {
        n = round_up(n);
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    int64_t size() const { return size_; }
    int64_t used() const { return used_; }
    int64_t peak() const { return peak_; }

  private:
    int64_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<int64_t, int64_t> free_;   // offset -> length
};

struct Req {
    int64_t id = 0;
    tacsl_request r{};
    bool render = false;          // a pose request: depth maps rendered on the device
    float* depth_map_out = nullptr;   // a pose request's rendered maps, if asked for
    std::vector<int32_t> obj, layout, sensor;
    int64_t n_taxel = 0, n_pixel = 0, n_image = 0, bytes = 0;
    Clock::time_point t_submit, t_done;
    bool done = false;
    int status = TACSL_OK;
};

// Bytes a request adds to a batch: inputs (pose 28, twist 24, parameters 16 per pad;
// depth 4 per pixel), outputs (28 per taxel, wrench 24 per pad, rgb 3 per pixel) and its
// workspace share (32 per pad; 16 per image: its first pixel, pad and object).
int64_t request_bytes(int64_t n_pad, int64_t n_taxel, int64_t n_pixel, int64_t n_image) {
    return n_pad * (28 + 24 + 16 + 24 + 32) + n_taxel * 28 + n_pixel * 7 + n_image * 16;
}
constexpr int64_t kBatchSlack = 16 * kGranule + 512;   // per-array alignment and the workspace header

struct Batch {
    std::vector<std::shared_ptr<Req>> reqs;
    bool render = false;               // pose requests: depth maps rendered on the device
    std::vector<CameraArgs> cams;      // the cameras when the batch was formed
    int stream = 0;
    int64_t off = -1, bytes = 0;
    Clock::time_point t_launch;
    bool timed_out = false;
};

class Server {
  public:
    ~Server() { stop(); }

    int create(const tacsl_server_config& cfg, const tacsl_sdf_set* sdfs, const tacsl_sensor_set* sensors,
               const float* taxels, int64_t n_points, int32_t n_layout, const int64_t* layout_first,
               const int32_t* layout_count) {
        cfg_ = cfg;
        int rc = build_table(sdfs, tab_);
        if (rc) return rc;
        if (sensors != nullptr) {
            if (sensors->models == nullptr || sensors->n_model < 1 || sensors->n_model > TACSL_MAX_MODEL)
                return fail(TACSL_ERR_INVALID_ARG, "sensor set: n_model outside [1, %d]", TACSL_MAX_MODEL);
            models_.assign(sensors->models, sensors->models + sensors->n_model);
            for (size_t m = 0; m < models_.size(); ++m) {
                const tacsl_sensor_model& sm = models_[m];
                if (sm.H < 4 || sm.W < 4 || sm.H % 4 || sm.W % 4 || sm.coeffs == nullptr || !aligned(sm.coeffs, 16))
                    return fail(TACSL_ERR_INVALID_ARG, "sensor model %d: bad size or coefficients", (int)m);
            }
        }
        if (taxels == nullptr || !aligned(taxels, 4) || n_points < 1)
            return fail(TACSL_ERR_INVALID_ARG, "taxel pool NULL, misaligned or empty");
        if (n_layout < 1 || layout_first == nullptr || layout_count == nullptr)
            return fail(TACSL_ERR_INVALID_ARG, "the server needs at least one taxel layout");
        layout_first_.assign(layout_first, layout_first + n_layout);
        layout_count_.assign(layout_count, layout_count + n_layout);
        for (int l = 0; l < n_layout; ++l)
            if (layout_count[l] < 1 || layout_count[l] > TACSL_MAX_TAXELS || layout_first[l] < 0 ||
                layout_first[l] + layout_count[l] > n_points)
                return fail(TACSL_ERR_INVALID_ARG, "layout %d outside the taxel pool", l);
        taxels_ = taxels;
        n_points_ = n_points;
        if ((rc = device_info(&dev_))) return rc;
        cudaError_t e = cudaGetDevice(&device_);
        if (e == cudaSuccess) e = cudaMalloc(&arena_ptr_, (size_t)cfg_.hbm_budget_bytes);
        if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "server arena of %lld bytes: %s",
                                          (long long)cfg_.hbm_budget_bytes, cudaGetErrorString(e));
        arena_.init(cfg_.hbm_budget_bytes);
        streams_.resize(cfg_.n_streams);
        events_.resize(cfg_.n_streams);
        busy_.assign(cfg_.n_streams, false);
        for (int s = 0; s < cfg_.n_streams; ++s) {
            e = cudaStreamCreateWithFlags(&streams_[s], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&events_[s], cudaEventDisableTiming);
            if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "server streams: %s", cudaGetErrorString(e));
        }
        running_ = true;
        worker_ = std::thread([this] { loop(); });
        return ok();
    }

    int set_cameras(const tacsl_camera* cams, int32_t n) {
        if (cams == nullptr) return fail(TACSL_ERR_INVALID_ARG, "cameras is NULL");
        if (n != static_cast<int32_t>(models_.size()))
            return fail(TACSL_ERR_INVALID_ARG, "%d cameras for %d sensor models", n, (int)models_.size());
        std::vector<CameraArgs> c(n);
        for (int m = 0; m < n; ++m) {
            const int rc = check_camera(&cams[m], c[m]);
            if (rc) return rc;
            if (c[m].H != models_[m].H || c[m].W != models_[m].W)
                return fail(TACSL_ERR_INVALID_ARG, "camera %d is %d x %d, sensor model %d is %d x %d", m, c[m].H, c[m].W,
                            m, models_[m].H, models_[m].W);
        }
        std::lock_guard<std::mutex> lk(mu_);
        cams_ = c;
        return ok();
    }

    int submit_poses(const tacsl_pose_request* q, int64_t* id) {
        if (q == nullptr || id == nullptr) return fail(TACSL_ERR_INVALID_ARG, "request or id is NULL");
        tacsl_request r{};
        r.n_pad = q->n_pad;
        r.obj_id = q->obj_id;
        r.layout = q->layout;
        r.sensor = q->sensor;
        r.pad_pose = q->pad_pose;
        r.pad_twist = q->pad_twist;
        r.k_n = q->k_n;
        r.k_d = q->k_d;
        r.k_t = q->k_t;
        r.mu = q->mu;
        r.depth = q->depth;
        r.f_n = q->f_n;
        r.f_t = q->f_t;
        r.wrench = q->wrench;
        r.rgb = q->rgb;
        return submit_any(&r, true, q->depth_map, id);
    }

    int submit(const tacsl_request* q, int64_t* id) {
        if (q == nullptr || id == nullptr) return fail(TACSL_ERR_INVALID_ARG, "request or id is NULL");
        return submit_any(q, false, nullptr, id);
    }

    int submit_any(const tacsl_request* q, bool render, float* depth_map_out, int64_t* id) {
        const int n = q->n_pad;
        if (n < 1) return fail(TACSL_ERR_INVALID_ARG, "a request needs at least one pad");
        if (n > cfg_.max_pads) return fail(TACSL_ERR_UNSUPPORTED, "request of %d pads > max_pads %d", n, cfg_.max_pads);
        if (q->obj_id == nullptr || q->layout == nullptr || q->sensor == nullptr || q->pad_pose == nullptr ||
            q->pad_twist == nullptr || q->k_n == nullptr || q->k_d == nullptr || q->k_t == nullptr ||
            q->mu == nullptr || (!render && (q->depth == nullptr || q->f_n == nullptr || q->f_t == nullptr)))
            return fail(TACSL_ERR_INVALID_ARG, "a required request array is NULL");
        auto r = std::make_shared<Req>();
        r->r = *q;
        r->render = render;
        r->depth_map_out = depth_map_out;
        r->obj.assign(q->obj_id, q->obj_id + n);
        r->layout.assign(q->layout, q->layout + n);
        r->sensor.assign(q->sensor, q->sensor + n);
        for (int b = 0; b < n; ++b) {
            if (r->obj[b] < 0 || r->obj[b] >= tab_.count)
                return fail(TACSL_ERR_INVALID_ARG, "pad %d: object %d not in the server's SDF set", b, r->obj[b]);
            if (r->layout[b] < 0 || r->layout[b] >= (int)layout_count_.size())
                return fail(TACSL_ERR_INVALID_ARG, "pad %d: layout %d out of range", b, r->layout[b]);
            if (r->sensor[b] < -1 || r->sensor[b] >= (int)models_.size())
                return fail(TACSL_ERR_INVALID_ARG, "pad %d: sensor %d out of range", b, r->sensor[b]);
            r->n_taxel += layout_count_[r->layout[b]];
            if (r->sensor[b] >= 0) {
                r->n_pixel += (int64_t)models_[r->sensor[b]].H * models_[r->sensor[b]].W;
                ++r->n_image;
            }
        }
        if (!render && r->n_image > 0 && (q->depth_map == nullptr || q->rgb == nullptr))
            return fail(TACSL_ERR_INVALID_ARG, "a request with images needs depth_map and rgb");
        if (render && r->n_image > 0) {
            std::lock_guard<std::mutex> lk(mu_);
            if (cams_.empty()) return fail(TACSL_ERR_INVALID_ARG, "a pose request with images needs the cameras set");
        }
        r->bytes = request_bytes(n, r->n_taxel, r->n_pixel, r->n_image);
        if (r->bytes + kBatchSlack > cfg_.hbm_budget_bytes)
            return fail(TACSL_ERR_UNSUPPORTED, "request needs %lld bytes, the budget is %lld", (long long)r->bytes,
                        (long long)cfg_.hbm_budget_bytes);
        {
            std::lock_guard<std::mutex> lk(mu_);
            r->id = next_id_++;
            r->t_submit = Clock::now();
            reqs_[r->id] = r;
            pending_.push_back(r);
            ++submitted_;
            *id = r->id;
        }
        cv_work_.notify_one();
        return ok();
    }

    int wait(int64_t id, int32_t timeout_ms, int32_t* status, double* latency_ms) {
        std::unique_lock<std::mutex> lk(mu_);
        auto it = reqs_.find(id);
        if (it == reqs_.end()) return fail(TACSL_ERR_INVALID_ARG, "unknown request %lld", (long long)id);
        std::shared_ptr<Req> r = it->second;
        auto done = [&] { return r->done; };
        if (timeout_ms < 0)
            cv_done_.wait(lk, done);
        else if (!cv_done_.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
            return fail(TACSL_ERR_TIMEOUT, "request %lld not finished after %d ms", (long long)id, timeout_ms);
        if (status) *status = r->status;
        if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
        reqs_.erase(id);
        return ok();
    }

    void stats(tacsl_server_stats* s) {
        std::lock_guard<std::mutex> lk(mu_);
        s->submitted = submitted_;
        s->completed = completed_;
        s->batches = batches_;
        s->pads_served = pads_served_;
        s->arena_bytes = arena_.size();
        s->arena_peak_bytes = arena_.peak();
        s->arena_used_bytes = arena_.used();
        s->max_batch_requests = max_batch_requests_;
        s->pending = static_cast<int32_t>(pending_.size());
    }

    void stop() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stopping_ = true;
        }
        cv_work_.notify_one();
        if (worker_.joinable()) worker_.join();
        for (size_t s = 0; s < streams_.size(); ++s) {
            if (streams_[s]) cudaStreamDestroy(streams_[s]);
            if (events_[s]) cudaEventDestroy(events_[s]);
        }
        streams_.clear();
        events_.clear();
        if (arena_ptr_) cudaFree(arena_ptr_);
        arena_ptr_ = nullptr;
    }

  private:
    void finish(Batch& bt, int status) {   // under mu_
        const auto now = Clock::now();
        for (auto& r : bt.reqs) {
            if (!r->done) {
                r->done = true;
                r->status = status;
                r->t_done = now;
                ++completed_;
            }
        }
        if (bt.off >= 0) arena_.release(bt.off, bt.bytes);
        busy_[bt.stream] = false;
    }

    // Oldest pending requests that fit now (under mu_); empty if the first does not.
    bool take_batch(Batch& bt) {
        const int64_t room = arena_.largest_free();
        int64_t bytes = kBatchSlack, pads = 0;
        const bool render = pending_.empty() ? false : pending_.front()->render;
        bt.render = render;
        bt.cams = cams_;
        while (!pending_.empty()) {
            const auto& r = pending_.front();
            if (r->render != render) break;   // a batch holds requests of one kind
            if (pads + r->r.n_pad > cfg_.max_pads || bytes + r->bytes > room) break;
            bytes += r->bytes;
            pads += r->r.n_pad;
            bt.reqs.push_back(r);
            pending_.pop_front();
        }
        if (bt.reqs.empty()) return false;
        bt.bytes = round_up(bytes);
        bt.off = arena_.alloc(bt.bytes);
        return true;   // the block fits: bytes <= the largest free block
    }

    // Plan, copy in, launch, copy out, record (outside mu_; the worker owns the stream).
    int launch(Batch& bt) {
        cudaStream_t st = streams_[bt.stream];
        std::vector<int32_t> obj, lay, sen;
        for (auto& r : bt.reqs) {
            obj.insert(obj.end(), r->obj.begin(), r->obj.end());
            lay.insert(lay.end(), r->layout.begin(), r->layout.end());
            sen.insert(sen.end(), r->sensor.begin(), r->sensor.end());
        }
        const int n = static_cast<int>(obj.size());
        tacsl_batch_desc d{n, obj.data(), lay.data(), sen.data(), static_cast<int32_t>(layout_count_.size()),
                           layout_first_.data(), layout_count_.data(), n_points_};
        tacsl_sensor_set ss{models_.data(), static_cast<int32_t>(models_.size())};
        tacsl_batch_plan plan;
        int rc = batch_plan(&d, models_.empty() ? nullptr : &ss, &plan, nullptr, nullptr);
        if (rc) return rc;
        // carve the block: workspace, inputs, outputs
        char* base = static_cast<char*>(arena_ptr_) + bt.off;
        int64_t at = 0;
        auto take = [&](int64_t nbytes) {
            char* p = base + at;
            at += round_up(std::max<int64_t>(nbytes, 1));
            return p;
        };
        void* ws = take(plan.workspace_bytes);
        float* pose = reinterpret_cast<float*>(take(4 * 7 * (int64_t)n));
        float* twist = reinterpret_cast<float*>(take(4 * 6 * (int64_t)n));
        float* prm[4];
        for (int k = 0; k < 4; ++k) prm[k] = reinterpret_cast<float*>(take(4 * (int64_t)n));
        float* dmap = reinterpret_cast<float*>(take(4 * plan.n_pixel_out));
        float* depth = reinterpret_cast<float*>(take(4 * plan.n_taxel_out));
        float* fn = reinterpret_cast<float*>(take(12 * plan.n_taxel_out));
        float* ft = reinterpret_cast<float*>(take(12 * plan.n_taxel_out));
        float* wrench = reinterpret_cast<float*>(take(24 * (int64_t)n));
        uint8_t* rgb = reinterpret_cast<uint8_t*>(take(3 * plan.n_pixel_out));
        if (at > bt.bytes) return fail(TACSL_ERR_CUDA, "server batch layout exceeds its block");   // not expected
        std::vector<unsigned char> host((size_t)plan.workspace_bytes);
        if ((rc = batch_pack(&plan, &d, host.data()))) return rc;
        auto copy = [&](void* dst, const void* src, int64_t nbytes, cudaMemcpyKind kind) {
            if (nbytes <= 0) return cudaSuccess;
            return cudaMemcpyAsync(dst, src, (size_t)nbytes, kind, st);
        };
        cudaError_t e = copy(ws, host.data(), plan.workspace_bytes, cudaMemcpyHostToDevice);
        int64_t p0 = 0, t0 = 0, q0 = 0;
        for (auto& r : bt.reqs) {
            const int64_t np = r->r.n_pad;
            const float* src[4] = {r->r.k_n, r->r.k_d, r->r.k_t, r->r.mu};
            if (e == cudaSuccess) e = copy(pose + 7 * p0, r->r.pad_pose, 28 * np, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = copy(twist + 6 * p0, r->r.pad_twist, 24 * np, cudaMemcpyHostToDevice);
            for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = copy(prm[k] + p0, src[k], 4 * np, cudaMemcpyHostToDevice);
            if (e == cudaSuccess && r->n_pixel > 0 && !bt.render)
                e = copy(dmap + q0, r->r.depth_map, 4 * r->n_pixel, cudaMemcpyHostToDevice);
            p0 += np;
            t0 += r->n_taxel;
            q0 += r->n_pixel;
        }
        if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "server copy-in: %s", cudaGetErrorString(e));
        tacsl_batch_io io{taxels_, pose, twist, depth, fn, ft, wrench, dmap, rgb};
        BatchCall c;
        c.tab = tab_;
        c.prm = Params4{prm[0], prm[1], prm[2], prm[3], n};
        c.dev = dev_;
        // a batch of pose requests renders its depth maps, and renders and shades only
        // if some request asks for the maps or the images
        bool want_rgb = !bt.render, want_map = false;
        for (auto& r : bt.reqs)
            if (r->n_pixel > 0) {
                want_rgb = want_rgb || r->r.rgb != nullptr;
                want_map = want_map || r->depth_map_out != nullptr;
            }
        if (bt.render && plan.n_image > 0 && (want_rgb || want_map) &&
            (rc = launch_batch_render(&plan, ws, tab_, bt.cams.data(), pose, dmap, st)))
            return rc;
        if (plan.n_image > 0 && want_rgb && (rc = launch_batch_shade(&plan, ws, &ss, &io, *dev_, 0, 0, st))) return rc;
        if ((rc = launch_batch_forces(&plan, ws, c.tab, c.prm, &io, *dev_, 4, true, st))) return rc;
        p0 = t0 = q0 = 0;
        for (auto& r : bt.reqs) {
            const int64_t np = r->r.n_pad;
            // (a pose request's outputs are optional: only those asked for travel back)
            if (e == cudaSuccess && r->r.depth) e = copy(r->r.depth, depth + t0, 4 * r->n_taxel, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && r->r.f_n) e = copy(r->r.f_n, fn + 3 * t0, 12 * r->n_taxel, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && r->r.f_t) e = copy(r->r.f_t, ft + 3 * t0, 12 * r->n_taxel, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && r->r.wrench) e = copy(r->r.wrench, wrench + 6 * p0, 24 * np, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && r->n_pixel > 0 && r->r.rgb)
                e = copy(r->r.rgb, rgb + 3 * q0, 3 * r->n_pixel, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && r->n_pixel > 0 && r->depth_map_out)
                e = copy(r->depth_map_out, dmap + q0, 4 * r->n_pixel, cudaMemcpyDeviceToHost);
            p0 += np;
            t0 += r->n_taxel;
            q0 += r->n_pixel;
        }
        if (e == cudaSuccess) e = cudaEventRecord(events_[bt.stream], st);
        if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "server copy-out: %s", cudaGetErrorString(e));
        return TACSL_OK;
    }

    void loop() {
        cudaSetDevice(device_);
        std::vector<Batch> inflight;
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            // 1. retire finished batches
            for (size_t i = 0; i < inflight.size();) {
                Batch& bt = inflight[i];
                const cudaError_t q = cudaEventQuery(events_[bt.stream]);
                if (q == cudaSuccess || q != cudaErrorNotReady) {
                    finish(bt, q == cudaSuccess ? (bt.timed_out ? TACSL_ERR_TIMEOUT : TACSL_OK) : TACSL_ERR_CUDA);
                    inflight.erase(inflight.begin() + i);
                    cv_done_.notify_all();
                    continue;
                }
                if (!bt.timed_out && Clock::now() - bt.t_launch > std::chrono::milliseconds(cfg_.batch_timeout_ms)) {
                    bt.timed_out = true;   // its requests fail now; its block waits for the GPU
                    const auto now = Clock::now();
                    for (auto& r : bt.reqs)
                        if (!r->done) {
                            r->done = true;
                            r->status = TACSL_ERR_TIMEOUT;
                            r->t_done = now;
                            ++completed_;
                        }
                    cv_done_.notify_all();
                }
                ++i;
            }
            // 2. new batches on free streams
            for (int s = 0; s < cfg_.n_streams && !pending_.empty(); ++s) {
                if (busy_[s]) continue;
                Batch bt;
                bt.stream = s;
                if (!take_batch(bt)) break;   // the oldest request waits for memory
                busy_[s] = true;
                ++batches_;
                max_batch_requests_ = std::max<int32_t>(max_batch_requests_, (int32_t)bt.reqs.size());
                for (auto& r : bt.reqs) pads_served_ += r->r.n_pad;
                lk.unlock();
                const int rc = launch(bt);
                lk.lock();
                bt.t_launch = Clock::now();
                if (rc != TACSL_OK) {
                    // nothing usable was queued after the failure point; wait for what was
                    cudaStreamSynchronize(streams_[s]);
                    finish(bt, rc);
                    cv_done_.notify_all();
                } else {
                    inflight.push_back(std::move(bt));
                }
            }
            if (stopping_ && pending_.empty() && inflight.empty()) break;
            if (inflight.empty())
                cv_work_.wait(lk, [&] { return stopping_ || !pending_.empty(); });
            else
                cv_work_.wait_for(lk, std::chrono::microseconds(20));
        }
        running_ = false;
    }

    tacsl_server_config cfg_{};
    SdfTable tab_{};
    std::vector<tacsl_sensor_model> models_;
    std::vector<CameraArgs> cams_;   // per sensor model, for pose requests (under mu_)
    std::vector<int64_t> layout_first_;
    std::vector<int32_t> layout_count_;
    const float* taxels_ = nullptr;
    int64_t n_points_ = 0;
    DevInfo* dev_ = nullptr;
    int device_ = 0;
    void* arena_ptr_ = nullptr;
    Arena arena_;
    std::vector<cudaStream_t> streams_;
    std::vector<cudaEvent_t> events_;
    std::vector<bool> busy_;
    std::mutex mu_;
    std::condition_variable cv_work_, cv_done_;
    std::deque<std::shared_ptr<Req>> pending_;
    std::map<int64_t, std::shared_ptr<Req>> reqs_;
    std::thread worker_;
    bool running_ = false, stopping_ = false;
    int64_t next_id_ = 1, submitted_ = 0, completed_ = 0, batches_ = 0, pads_served_ = 0;
    int32_t max_batch_requests_ = 0;
};

}  // namespace serve
}  // namespace tacsl

extern "C" {

int tacsl_server_create(const tacsl_server_config* config, const tacsl_sdf_set* sdfs, const tacsl_sensor_set* sensors,
                        const float* taxels, int64_t n_points, int32_t n_layout, const int64_t* layout_first,
                        const int32_t* layout_count, tacsl_server_t* server) {
    using namespace tacsl;
    if (server == nullptr || config == nullptr) return fail(TACSL_ERR_INVALID_ARG, "config or server is NULL");
    *server = nullptr;
    if (config->hbm_budget_bytes < (int64_t(1) << 20))
        return fail(TACSL_ERR_INVALID_ARG, "hbm_budget_bytes = %lld < 1 MiB", (long long)config->hbm_budget_bytes);
    if (config->max_pads < 1) return fail(TACSL_ERR_INVALID_ARG, "max_pads = %d < 1", config->max_pads);
    if (config->n_streams < 1 || config->n_streams > 8)
        return fail(TACSL_ERR_INVALID_ARG, "n_streams = %d outside [1, 8]", config->n_streams);
    if (config->batch_timeout_ms < 1) return fail(TACSL_ERR_INVALID_ARG, "batch_timeout_ms must be >= 1");
    auto* s = new serve::Server();
    const int rc = s->create(*config, sdfs, sensors, taxels, n_points, n_layout, layout_first, layout_count);
    if (rc) {
        delete s;
        return rc;
    }
    *server = reinterpret_cast<tacsl_server_t>(s);
    return ok();
}

int tacsl_server_submit(tacsl_server_t server, const tacsl_request* request, int64_t* request_id) {
    if (server == nullptr) return fail(TACSL_ERR_INVALID_ARG, "server is NULL");
    return reinterpret_cast<tacsl::serve::Server*>(server)->submit(request, request_id);
}

int tacsl_server_wait(tacsl_server_t server, int64_t request_id, int32_t timeout_ms, int32_t* status,
                      double* latency_ms) {
    if (server == nullptr) return fail(TACSL_ERR_INVALID_ARG, "server is NULL");
    return reinterpret_cast<tacsl::serve::Server*>(server)->wait(request_id, timeout_ms, status, latency_ms);
}

int tacsl_server_set_cameras(tacsl_server_t server, const tacsl_camera* cameras, int32_t n_camera) {
    if (server == nullptr) return fail(TACSL_ERR_INVALID_ARG, "server is NULL");
    return reinterpret_cast<tacsl::serve::Server*>(server)->set_cameras(cameras, n_camera);
}

int tacsl_server_submit_poses(tacsl_server_t server, const tacsl_pose_request* request, int64_t* request_id) {
    if (server == nullptr) return fail(TACSL_ERR_INVALID_ARG, "server is NULL");
    return reinterpret_cast<tacsl::serve::Server*>(server)->submit_poses(request, request_id);
}

int tacsl_server_get_stats(tacsl_server_t server, tacsl_server_stats* stats) {
    if (server == nullptr || stats == nullptr) return fail(TACSL_ERR_INVALID_ARG, "server or stats is NULL");
    reinterpret_cast<tacsl::serve::Server*>(server)->stats(stats);
    return ok();
}

int tacsl_server_destroy(tacsl_server_t server) {
    if (server == nullptr) return ok();
    delete reinterpret_cast<tacsl::serve::Server*>(server);
    return ok();
}

}  // extern "C"
