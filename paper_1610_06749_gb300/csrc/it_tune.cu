// it_tune.cu -- native autotuner of the step kernel's launch shape.
//
// Candidates: the simple kernel; the z-march kernel over tile heights that
// give each thread one or two float4 items, 1 or 2 CTAs per SM, ring depths
// 3..8 and the two grid rules (one CTA per resident slot, or a multiple of
// the tile count); and the two-steps-per-launch z-march kernel over 1 or 2
// CTAs per SM, ring depths 3..6 and the two grid rules.  Each candidate is
// timed with CUDA events on the context stream over a few steps of the live
// state, which is saved before and restored after every trial.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "it_internal.cuh"

namespace itk {

namespace {

struct Shape {
    int kernel, ty, cps, s, grid;
};

using Key = std::tuple<int, int, int, int, int>;
std::map<Key, Shape> g_cache;
std::mutex g_cache_mu;

std::vector<Shape> candidates(const it_ctx *c) {
    std::vector<Shape> v;
    v.push_back({IT_KERNEL_SIMPLE, 0, 0, 0, 0});
    const int nx = c->g.nx, ny = c->g.ny;
    if (c->prec != IT_FP32 || nx % 4 != 0 || (nx > 256 && nx % 256 != 0)) return v;
    const int ncol4 = nx / 4;
    for (int cps = 1; cps <= 2; ++cps) {
        const int threads = cps == 1 ? 512 : 256;
        for (int ty = 1; ty <= std::min(ny, 255); ++ty) {
            if (ny % ty) continue;
            const int items = ncol4 * ty;
            if (2 * items < threads || items > 2 * threads) continue;   // 0.5 .. 2 items per thread
            for (int s : {3, 4, 5, 6, 8})
                for (int grid : {0, -1}) v.push_back({IT_KERNEL_ZMARCH, ty, cps, s, grid});
        }
    }
    // two steps per launch: one float4 per thread, so the tile height is
    // threads / (nx/4)
    for (int cps = 1; cps <= 2; ++cps) {
        const int threads = cps == 1 ? 512 : 256;
        if (threads % ncol4 != 0 || 2 * ncol4 > threads) continue;
        const int ty = threads / ncol4;
        if (ny % ty != 0 || ny < 4) continue;
        for (int s : {3, 4, 5, 6})
            for (int grid : {0, -1}) v.push_back({IT_KERNEL_ZMARCH2, ty, cps, s, grid});
    }
    return v;
}

int time_shape(it_ctx *c, const Shape &sh, int trial, const void *backup, size_t bytes, double *us) {
    int rc = set_launch(c, sh.kernel, sh.ty, sh.cps, sh.s, sh.grid);
    if (rc) return rc;
    if (c->kernel != sh.kernel) return IT_EINVAL;
    cudaEvent_t e0, e1;
    IT_CK(cudaEventCreate(&e0));
    IT_CK(cudaEventCreate(&e1));
    const int cur = c->cur;
    // one launch: one step, or two with the two-step kernel (trial is even)
    auto launch = [&]() {
        return c->kernel == IT_KERNEL_ZMARCH    ? launch_step_zmarch(c, c->stream)
               : c->kernel == IT_KERNEL_ZMARCH2 ? launch_step_zmarch2(c, c->stream)
                                                : launch_step_simple(c, c->stream);
    };
    const int per = c->kernel == IT_KERNEL_ZMARCH2 ? 2 : 1;
    for (int q = 0; q < 2 && rc == IT_OK; q += per) rc = launch();
    cudaEventRecord(e0, c->stream);
    for (int q = 0; q < trial && rc == IT_OK; q += per) rc = launch();
    cudaEventRecord(e1, c->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // back to the saved state (an even number of steps keeps the same set)
    c->cur = cur;
    const char *b = (const char *)backup;
    cudaMemcpyAsync(c->n[cur][0], b, bytes, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(c->n[cur][1], b + bytes, bytes, cudaMemcpyDeviceToDevice, c->stream);
    int errflag = 0;
    cudaMemcpyAsync(&errflag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
    if (errflag) {
        cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
        return IT_ETIMEOUT;
    }
    *us = 1e3 * ms / trial;
    return IT_OK;
}

}  // namespace

}  // namespace itk

using namespace itk;

extern "C" int it_autotune(it_ctx *c, int trial_steps, int flags, double *best_us) {
    if (!c) {
        set_error("ctx is NULL");
        return IT_EINVAL;
    }
    if (c->steps != 0) {
        set_error("autotune only before the first step");
        return IT_ESTATE;
    }
    int trial = trial_steps > 0 ? trial_steps : 8;
    trial += trial & 1;
    const Key key{c->g.nx, c->g.ny, c->g.nz, c->prec, c->p.lateral_bc};
    if (!(flags & 1)) {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            const Shape sh = it->second;
            int rc = set_launch(c, sh.kernel, sh.ty, sh.cps, sh.s, sh.grid);
            if (rc == IT_OK) {
                if (best_us) *best_us = -1.0;
                return IT_OK;
            }
        }
    }
    const size_t bytes = c->g.cells() * c->esize;
    void *backup = nullptr;
    IT_CK(cudaMalloc(&backup, 2 * bytes));
    IT_CK(cudaMemcpyAsync(backup, c->n[c->cur][0], bytes, cudaMemcpyDeviceToDevice, c->stream));
    IT_CK(cudaMemcpyAsync((char *)backup + bytes, c->n[c->cur][1], bytes, cudaMemcpyDeviceToDevice, c->stream));
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    Shape best{IT_KERNEL_SIMPLE, 0, 0, 0, 0};
    double best_t = 1e300;
    for (const Shape &sh : candidates(c)) {
        double us = 0.0;
        if (time_shape(c, sh, trial, backup, bytes, &us) == IT_OK && us < best_t) {
            best_t = us;
            best = sh;
        }
    }
    cudaFree(backup);
    int rc = set_launch(c, best.kernel, best.ty, best.cps, best.s, best.grid);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        g_cache[key] = best;
    }
    set_error("");
    if (best_us) *best_us = best_t;
    return IT_OK;
}
