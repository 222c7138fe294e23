// Batched scans (twa_batch_run): many (N, alpha, w) points advanced together by
// grouped persistent launches, replayed as CUDA graphs, with tile shapes from a
// built-in autotuner.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "twa_internal.cuh"

namespace {

// Device copy of a context's trajectories and window sums (autotuning trials
// advance the state; it is put back afterwards). The buffers come from the
// context's allocator and are returned by release() on every path.
struct Snapshot {
    twa_ctx* owner = nullptr;
    float *X = nullptr, *Y = nullptr, *Z = nullptr;
    double* mom = nullptr;
    int64_t t = 0, count = 0;
    bool taken = false;   // the copies completed: restore() may put them back

    void release() {
        if (owner) {
            void* p[] = {X, Y, Z, mom};
            for (void* q : p) twa::dev_free(owner, q);
        }
        X = Y = Z = nullptr;
        mom = nullptr;
        taken = false;
    }
    Snapshot() = default;
    Snapshot(const Snapshot&) = delete;
    Snapshot& operator=(const Snapshot&) = delete;
    ~Snapshot() { release(); }
};

int snapshot(twa_ctx* c, Snapshot& s) {
    s.release();
    s.owner = c;
    const size_t mn = sizeof(float) * c->M * c->N;
    if (twa::dev_malloc(c, &s.X, mn) != cudaSuccess || twa::dev_malloc(c, &s.Y, mn) != cudaSuccess ||
        twa::dev_malloc(c, &s.Z, mn) != cudaSuccess ||
        twa::dev_malloc(c, &s.mom, sizeof(double) * 5 * c->M) != cudaSuccess) {
        s.release();
        return twa::set_error(c, TWA_ENOMEM, "batch autotuner: device allocation of the snapshot");
    }
    twa::TcState* t = c->tc;
    cudaError_t e = cudaMemcpyAsync(s.X, t->X, mn, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.Y, t->Y, mn, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.Z, t->Z, mn, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s.mom, c->mom, sizeof(double) * 5 * c->M, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&s.t, c->d_t, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&s.count, c->d_count, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(c->stream);   // no copy may still write into the buffers freed below
        s.release();
        return twa::cuda_check(c, e, "batch autotuner: snapshot copy");
    }
    s.taken = true;
    return TWA_OK;
}

// Put the snapshot back (and release it).
int restore(twa_ctx* c, Snapshot& s) {
    if (!s.taken) {
        s.release();
        return TWA_OK;
    }
    const size_t mn = sizeof(float) * c->M * c->N;
    twa::TcState* t = c->tc;
    cudaError_t e = cudaMemcpyAsync(t->X, s.X, mn, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->Y, s.Y, mn, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->Z, s.Z, mn, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->mom, s.mom, sizeof(double) * 5 * c->M, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_t, &s.t, sizeof(int64_t), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_count, &s.count, sizeof(int64_t), cudaMemcpyHostToDevice, c->stream);
    int rc = (e == cudaSuccess) ? twa::tc_state_changed(c)   // images and partial sums of the restored state
                                : twa::cuda_check(c, e, "batch autotuner: restore copy");
    const cudaError_t es = cudaStreamSynchronize(c->stream);
    if (!rc && es != cudaSuccess) rc = twa::cuda_check(c, es, "batch autotuner: restore");
    s.release();
    return rc;
}

int set_tiles_all(std::vector<twa_ctx*>& ctx, int bn, int kc) {
    for (twa_ctx* c : ctx) {
        int rc = twa::tc_set_tiles(c, bn, kc);
        if (rc) return rc;
    }
    return TWA_OK;
}

// Time `steps` grouped steps of all contexts (ms per step, CUDA events).
int time_batch(std::vector<twa_ctx*>& ctx, int steps, float* ms) {
    twa_ctx* lead = ctx[0];
    twa::TcBatch* b = nullptr;
    int rc = twa::tc_batch_build(ctx.data(), (int)ctx.size(), lead, &b);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // the contexts sit at step 0 (trials run between snapshot and restore)
    rc = twa::tc_batch_prime(lead, b, 0);
    if (!rc) rc = twa::tc_batch_step(lead, b, 0);   // untimed: first launch of this configuration
    cudaEventRecord(e0, lead->stream);
    for (int s = 1; s <= steps && !rc; ++s) rc = twa::tc_batch_step(lead, b, s);
    cudaEventRecord(e1, lead->stream);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(ms, e0, e1);
    *ms /= steps;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    twa::tc_batch_free(b);
    return rc;
}

// Pick the fastest compiled tile configuration for this batch. Every context is
// put back to its snapshot before returning, also when a trial fails.
int autotune(std::vector<twa_ctx*>& ctx, int* bn, int* kc) {
    // the one-operand rings (KC = 3, 4) are candidates for the precisions with at
    // most two products per entry
    const bool one_b = ctx[0]->tc->terms <= 2 && ctx[0]->tc->lterms <= 2;
    std::vector<std::pair<int, int>> cand = {{256, 1}, {192, 1}, {256, 0}, {128, 1}};
    if (ctx[0]->tc->pair) cand = {{256, 0}, {256, 1}};   // the configurations compiled for CTA pairs (default)
    if (one_b) {
        cand.push_back({256, 3});
        cand.push_back({256, 4});
    }
    std::vector<Snapshot> snap(ctx.size());
    const int bn0 = *bn, kc0 = *kc;
    auto put_back = [&](int rc) {
        // restore what was snapshotted (a failed trial leaves the state advanced)
        for (size_t p = 0; p < ctx.size(); ++p) {
            const int r = restore(ctx[p], snap[p]);
            if (!rc) rc = r;
        }
        return rc;
    };
    for (size_t p = 0; p < ctx.size(); ++p) {
        int rc = snapshot(ctx[p], snap[p]);
        if (rc) return put_back(rc);
    }
    float best = INFINITY;
    for (auto& cd : cand) {
        int rc = set_tiles_all(ctx, cd.first, cd.second);
        float ms = 0.f;
        if (!rc) rc = time_batch(ctx, 5, &ms);
        if (rc) {
            // back to the configuration the contexts had before the trials
            set_tiles_all(ctx, bn0, kc0);
            return put_back(rc);
        }
        if (ms < best) {
            best = ms;
            *bn = cd.first;
            *kc = cd.second;
        }
    }
    const int rc = put_back(TWA_OK);
    if (rc) return rc;
    return set_tiles_all(ctx, *bn, *kc);
}

// Run steps t0 .. t0 + reps - 1 of the running points as replays of the
// captured step of each parity. At t0 = 0 the noise part of the first step is
// computed first; later stages find it in place (the previous stage's last step
// computed it for every point, the finished ones included).
int run_stage(std::vector<twa_ctx*>& active, int64_t t0, int64_t reps, cudaStream_t cap) {
    twa_ctx* lead = active[0];
    twa::TcBatch* b = nullptr;
    int rc = twa::tc_batch_build(active.data(), (int)active.size(), lead, &b);
    if (rc) return rc;
    if (t0 == 0 && (rc = twa::tc_batch_prime(lead, b, 0))) {
        twa::tc_batch_free(b);
        return rc;
    }
    cudaStream_t saved = lead->stream;
    cudaGraph_t g[2] = {nullptr, nullptr};
    cudaGraphExec_t ge[2] = {nullptr, nullptr};
    lead->stream = cap;
    bool graph = true;
    for (int k = 0; k < 2 && graph; ++k) {
        const int64_t t = t0 + k;
        graph = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (graph) {
            rc = twa::tc_batch_step(lead, b, t);
            graph = cudaStreamEndCapture(cap, &g[k]) == cudaSuccess && rc == TWA_OK &&
                    cudaGraphInstantiate(&ge[k], g[k], 0) == cudaSuccess;
        }
    }
    lead->stream = saved;
    cudaGetLastError();
    rc = TWA_OK;
    for (int64_t s = 0; s < reps && rc == TWA_OK; ++s) {
        const int64_t t = t0 + s;
        if (graph) {
            if (cudaGraphLaunch(ge[(t - t0) & 1], lead->stream) != cudaSuccess)
                rc = twa::set_error(lead, TWA_ECUDA, "cudaGraphLaunch");
        } else {
            rc = twa::tc_batch_step(lead, b, t);   // capture unavailable: launch directly
        }
    }
    if (cudaStreamSynchronize(lead->stream) != cudaSuccess && rc == TWA_OK)
        rc = twa::set_error(lead, TWA_ECUDA, "batch stage failed");
    for (int k = 0; k < 2; ++k) {
        if (ge[k]) cudaGraphExecDestroy(ge[k]);
        if (g[k]) cudaGraphDestroy(g[k]);
    }
    twa::tc_batch_free(b);
    return rc;
}

}  // namespace

extern "C" int twa_batch_run(const twa_point* pts, int n, int64_t M, uint64_t seed, const twa_opts* opts,
                             twa_obs* out, int* tiles) {
    using twa::set_error;
    twa::NvtxRange range("twa_batch_run");
    if (!pts || !out || n < 1 || n > 65536) return set_error(nullptr, TWA_EINVAL, "twa_batch_run: bad points or n");
    if (M < 1 || M > (int64_t)1 << 30) return set_error(nullptr, TWA_EINVAL, "twa_batch_run: M must be in [1, 2^30]");
    twa_opts o;
    twa_opts_default(&o);
    o.precision = TWA_PREC_BF16X3;
    if (opts) o = *opts;
    const bool resident = o.ws_route == TWA_ROUTE_RESIDENT;
    if (resident) {
        // every point's whole run in one launch per CTA shape (FP32 SIMT), or in
        // one launch on the tensor cores (BF16X2, N <= 128)
        if (o.precision != TWA_PREC_FP32 && o.precision != TWA_PREC_BF16X2)
            return set_error(nullptr, TWA_EUNSUPPORTED,
                             "twa_batch_run: the resident route runs in TWA_PREC_FP32 or TWA_PREC_BF16X2");
        const int64_t nmax = o.precision == TWA_PREC_BF16X2 ? TWA_RESIDENT_TC_MAX_N : TWA_RESIDENT_MAX_N;
        for (int p = 0; p < n; ++p)
            if (pts[p].N > nmax)
                return set_error(nullptr, TWA_EUNSUPPORTED, "twa_batch_run: N too large for the resident route");
    } else {
        if (o.precision != TWA_PREC_BF16 && o.precision != TWA_PREC_BF16X3 && o.precision != TWA_PREC_BF16X2 &&
            o.precision != TWA_PREC_BF16L2 && o.precision != TWA_PREC_BF16B)
            return set_error(nullptr, TWA_EUNSUPPORTED, "twa_batch_run: batches run on the BF16 precision paths");
        o.ws_route = TWA_ROUTE_DENSE;
    }
    o.noise_route = TWA_NOISE_CHOLESKY;
    for (int p = 0; p < n; ++p)
        if (pts[p].steps < 1 || pts[p].steps > 0xFFFFFFFFll)
            return set_error(nullptr, TWA_EINVAL, "twa_batch_run: every point needs 1 <= steps < 2^32");
    std::vector<twa_ctx*> ctx(n, nullptr);
    auto cleanup = [&](int rc) {
        for (twa_ctx* c : ctx) twa_destroy(c);
        return rc;
    };
    int rc;
    // Set-up (pump matrix, Cholesky factor, Lanczos bounds, initial state) is a
    // chain of small dependent kernels per point: the points are set up from
    // several host threads, each on a stream of its own, so that the chains
    // overlap on the GPU. Afterwards every context works on the caller's stream.
    {
        int dev = 0;
        cudaGetDevice(&dev);
        const int nw = n < 16 ? n : 16;
        std::vector<cudaStream_t> streams(nw, nullptr);
        std::vector<int> rcs(n, TWA_OK);
        std::vector<std::string> errs(n);
        bool ok = true;
        for (int w = 0; w < nw && ok; ++w)
            ok = cudaStreamCreateWithFlags(&streams[w], cudaStreamNonBlocking) == cudaSuccess;
        if (ok) {
            std::atomic<int> next{0};
            auto worker = [&](int w) {
                cudaSetDevice(dev);
                for (int p; (p = next.fetch_add(1)) < n;) {
                    twa_opts op = o;
                    op.window_start = pts[p].window_start;
                    // a caller's allocator may tie its blocks to the stream they were
                    // allocated on: then every point is set up on the caller's stream
                    op.stream = o.alloc ? o.stream : streams[w];
                    int r = twa_init(&ctx[p], pts[p].N, pts[p].alpha, pts[p].w, pts[p].Gamma, pts[p].dt, seed, &op);
                    if (r) {
                        rcs[p] = r;
                        errs[p] = twa_last_error(nullptr);
                        continue;
                    }
                    r = twa_run(ctx[p], M, 0);
                    if (!r && cudaStreamSynchronize(streams[w]) != cudaSuccess) r = TWA_ECUDA;
                    if (r) {
                        rcs[p] = r;
                        errs[p] = ctx[p]->err;
                    }
                }
            };
            std::vector<std::thread> pool;
            for (int w = 0; w < nw; ++w) pool.emplace_back(worker, w);
            for (auto& th : pool) th.join();
        }
        for (int p = 0; p < n; ++p)
            if (ctx[p]) ctx[p]->stream = (cudaStream_t)o.stream;
        for (cudaStream_t st : streams)
            if (st) cudaStreamDestroy(st);
        if (!ok) {
            set_error(nullptr, TWA_ECUDA, "twa_batch_run: cudaStreamCreate");
            return cleanup(TWA_ECUDA);
        }
        for (int p = 0; p < n; ++p)
            if (rcs[p]) {
                set_error(nullptr, rcs[p], errs[p]);
                return cleanup(rcs[p]);
            }
    }
    twa_ctx* lead = ctx[0];
    if (resident) {
        std::vector<int64_t> steps(n);
        for (int p = 0; p < n; ++p) steps[p] = pts[p].steps;
        if ((rc = twa::res_run_many(ctx.data(), steps.data(), n, lead, (cudaStream_t)o.stream))) {
            set_error(nullptr, rc, lead->err);
            return cleanup(rc);
        }
        if (tiles) tiles[0] = tiles[1] = 0;   // no tensor-core tiles on this route
        for (int p = 0; p < n; ++p) {
            ctx[p]->steps = pts[p].steps;
            if ((rc = twa_observables(ctx[p], &out[p])) ||
                (pts[p].means && (rc = twa_get_moments(ctx[p], pts[p].means, 0)))) {
                set_error(nullptr, rc, ctx[p]->err);
                return cleanup(rc);
            }
        }
        return cleanup(TWA_OK);
    }
    int bn = lead->tc->bn, kc = lead->tc->kc;
    if (!getenv("TWA_TC_BN") && !getenv("TWA_TC_KC")) {
        // tune on the points of the stage with the most work (steps x N^2 of the
        // points still running), which dominates the run
        std::vector<int64_t> cuts;
        for (int p = 0; p < n; ++p) cuts.push_back(pts[p].steps);
        std::sort(cuts.begin(), cuts.end());
        int64_t prev = 0, best_end = cuts.back();
        double best_work = -1.0;
        for (int64_t end : cuts) {
            if (end == prev) continue;
            double w = 0.0;
            for (int p = 0; p < n; ++p)
                if (pts[p].steps >= end) w += (double)pts[p].N * (double)pts[p].N;
            w *= (double)(end - prev);
            if (w > best_work) best_work = w, best_end = end;
            prev = end;
        }
        std::vector<twa_ctx*> trial;
        for (int p = 0; p < n; ++p)
            if (pts[p].steps >= best_end) trial.push_back(ctx[p]);
        if ((rc = autotune(trial, &bn, &kc)) || (rc = set_tiles_all(ctx, bn, kc))) {
            set_error(nullptr, rc, lead->err);
            return cleanup(rc);
        }
    }
    if (tiles) {
        tiles[0] = bn;
        tiles[1] = kc;
    }
    // stages: the running set shrinks as points reach their step counts
    std::vector<int64_t> ends;
    for (int p = 0; p < n; ++p) ends.push_back(pts[p].steps);
    std::sort(ends.begin(), ends.end());
    ends.erase(std::unique(ends.begin(), ends.end()), ends.end());
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
        set_error(nullptr, TWA_ECUDA, "twa_batch_run: cudaStreamCreate");
        return cleanup(TWA_ECUDA);
    }
    int64_t done = 0;
    for (int64_t end : ends) {
        std::vector<int> idx;
        for (int p = 0; p < n; ++p)
            if (pts[p].steps > done) idx.push_back(p);
        // largest problems first in the tile list
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return pts[a].N > pts[b].N; });
        std::vector<twa_ctx*> active;
        for (int p : idx) active.push_back(ctx[p]);
        if ((rc = run_stage(active, done, end - done, cap))) {
            set_error(nullptr, rc, active[0]->err);
            cudaStreamDestroy(cap);
            return cleanup(rc);
        }
        done = end;
    }
    cudaStreamDestroy(cap);
    for (int p = 0; p < n; ++p) {
        ctx[p]->steps = pts[p].steps;
        if ((rc = twa_observables(ctx[p], &out[p])) ||
            (pts[p].means && (rc = twa_get_moments(ctx[p], pts[p].means, 0)))) {
            set_error(nullptr, rc, ctx[p]->err);
            return cleanup(rc);
        }
    }
    return cleanup(TWA_OK);
}
