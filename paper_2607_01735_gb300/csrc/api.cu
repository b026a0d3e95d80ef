// C ABI entry points of librbgs (declared in include/rbgs.h): context life cycle,
// layout staging, sweep scheduling (one cooperative launch for all sweeps, direct
// launches, a cached CUDA graph, temporally blocked passes, or one cluster launch for the
// FP32 inner sweeps of small grids), residual evaluation, the convergence loop and the
// mixed-precision refinement loop.
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "sweep_impl.cuh"

namespace rbgs {

namespace {
thread_local char g_err[1024] = "";
}

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = '\0'; }

namespace {

constexpr int kMaxN = 1 << 18;
constexpr long kGraphSweeps = 32;    // sweeps per cached graph
constexpr int kGraphMaxN = 2048;     // graphs pay off where launches dominate
// FP64 sweeps in one cooperative launch (persistent.cu) for kPersistMinN <= n <= kPersistMaxN.
// Measured on GB300 against one launch per colour (graphs up to 2048): 0.94x at 383^2,
// 1.15x at 511^2, 1.29x at 1023^2, 1.32x at 4095^2, 1.10x at 16383^2; below ~400 the grid
// barrier costs more than a graph's launches.  Above 32768 its flattened item index would
// leave 32 bits.
constexpr int kPersistMinN = 416;
// FP32 inner sweeps in one launch of one 16-block cluster (cluster_sweeps.cu) up to this
// size.  Measured on GB300 against cached graphs of one launch per colour: 1.42x at 63^2,
// 1.46x at 127^2, 0.93x at 255^2, 0.49x at 511^2 (16 SMs do not match the whole GPU there).
constexpr int kClusterMaxN = 160;
constexpr int kPersistMaxN = 1 << 15;
// Fused update (opts.fma = 1): sweeps per block of one fixed-point scale.  The scale bounds
// max |u| + (sweeps) max |h2 f| / 2 a priori, so shorter blocks keep it tighter; the
// rescaling pass (max |u|, h2 f onto the grid: about one sweep's traffic) repeats per block.
constexpr long kFusedChunk = 1024;
// Residual checks without a new minimum of rho after which a solve stops (opts.stall_checks 0).
constexpr int kDefaultStallChecks = 64;

bool use_persistent(const rbgs_ctx *c) { return c->kernel == RBGS_KERNEL_PERSISTENT; }

bool device_accessible(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device-readable natural-layout view of a caller buffer: the pointer itself when the
// GPU can read it, else a copy in the context's staging buffer (stream-ordered).
rbgs_status stage_in(rbgs_ctx *c, const double *src, size_t count, const double **view) {
    if (device_accessible(src)) {
        *view = src;
        return RBGS_OK;
    }
    if (!c->staging) {
        size_t nat = (size_t)c->g.rows * c->g.rows;
        if (cudaMalloc(&c->staging, nat * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc of the %zu-byte staging buffer failed", nat * sizeof(double));
            return RBGS_ENOMEM;
        }
    }
    RBGS_CUDA(cudaMemcpyAsync(c->staging, src, count * sizeof(double), cudaMemcpyDefault, c->stream));
    *view = c->staging;
    return RBGS_OK;
}

// Packs device-readable natural-layout inputs into the context (f may be NULL: keep h2 f)
// and reduces ||h^2 b||^2 into dsum[1], all on c->stream.
rbgs_status enqueue_pack(rbgs_ctx *c, const double *f_view, const double *u_view) {
    const Geometry &g = c->g;
    c->black_fresh = false;
    rbgs_status st;
    if (f_view && (st = launch_pack_f(g, c->h2, f_view, c->f64.hf[0], c->f64.hf[1], c->stream)) != RBGS_OK) return st;
    if ((st = launch_pack_u(g, u_view, c->f64.u[0], c->f64.u[1], c->stream)) != RBGS_OK) return st;
    if (f_view && c->fused && (st = launch_fused_rhs_max(c, c->stream)) != RBGS_OK) return st;
    // ||h^2 b||^2 depends on f and the ring
    return launch_rhs_norm(c, c->stream);
}

rbgs_status load_problem(rbgs_ctx *c, const double *f, const double *u_init) {
    const Geometry &g = c->g;
    const double *fview = nullptr, *uview = nullptr;
    rbgs_status st;
    if (f && (st = stage_in(c, f, (size_t)g.n * g.n, &fview)) != RBGS_OK) return st;
    if (f && fview == c->staging) {
        // f goes through the staging buffer: pack it before u_init reuses the buffer
        if ((st = launch_pack_f(g, c->h2, fview, c->f64.hf[0], c->f64.hf[1], c->stream)) != RBGS_OK) return st;
        if (c->fused && (st = launch_fused_rhs_max(c, c->stream)) != RBGS_OK) return st;
        fview = nullptr;
    }
    if ((st = stage_in(c, u_init, (size_t)g.rows * g.rows, &uview)) != RBGS_OK) return st;
    if ((st = enqueue_pack(c, fview, uview)) != RBGS_OK) return st;
    RBGS_CUDA(cudaMemcpyAsync(c->hsum + 1, c->dsum + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    RBGS_CUDA(cudaStreamSynchronize(c->stream));
    c->den2 = c->hsum[1];
    return RBGS_OK;
}

void free_ctx(rbgs_ctx *c) {
    if (!c) return;
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->graph32) cudaGraphExecDestroy(c->graph32);
    for (int q = 0; q < 2; ++q) {
        cudaFree(c->f64.u[q]);
        cudaFree(c->f64.hf[q]);
        cudaFree(c->f64.alt[q]);
        cudaFree(c->f32.u[q]);
        cudaFree(c->f32.hf[q]);
        cudaFree(c->f32.alt[q]);
    }
    cudaFree(c->hq[0]);
    cudaFree(c->hq[1]);
    cudaFree(c->fwords);
    for (int q = 0; q < 2; ++q) {
        cudaFree(c->sin_f[q]);
        cudaFree(c->sin_u[q]);
        cudaFree(c->sout[q]);
        if (c->ev_copied[q]) cudaEventDestroy(c->ev_copied[q]);
        if (c->ev_packed[q]) cudaEventDestroy(c->ev_packed[q]);
        if (c->ev_unpacked[q]) cudaEventDestroy(c->ev_unpacked[q]);
        if (c->ev_out[q]) cudaEventDestroy(c->ev_out[q]);
    }
    if (c->h2d) cudaStreamDestroy(c->h2d);
    if (c->d2h) cudaStreamDestroy(c->d2h);
    cudaFree(c->dres);
    if (c->hres) cudaFreeHost(c->hres);
    cudaFree(c->staging);
    cudaFree(c->partials);
    cudaFree(c->dsum);
    cudaFree(c->dstatus);
    cudaFree(c->pcounter);
    if (c->hsum) cudaFreeHost(c->hsum);
    if (c->hstatus) cudaFreeHost(c->hstatus);
    if (c->capture) cudaStreamDestroy(c->capture);
    delete c;
}

// Zero-filled device buffer of `bytes` (stream-ordered fill).
rbgs_status alloc_zero(void **p, size_t bytes, cudaStream_t s) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("cudaMalloc of %zu bytes failed", bytes);
        return RBGS_ENOMEM;
    }
    RBGS_CUDA(cudaMemsetAsync(*p, 0, bytes, s));
    return RBGS_OK;
}

rbgs_status ensure_f64_alt(rbgs_ctx *c) {
    if (c->f64.alt[0]) return RBGS_OK;
    const size_t bytes = c->g.colour_elems() * sizeof(double);
    for (int q = 0; q < 2; ++q) {
        rbgs_status st = alloc_zero(reinterpret_cast<void **>(&c->f64.alt[q]), bytes, c->stream);
        if (st != RBGS_OK) return st;
    }
    c->f64.maps_ready = false;
    return RBGS_OK;
}

// FP32 correction, scaled defect and (for the temporal inner kernel) the partner buffers.
rbgs_status ensure_f32(rbgs_ctx *c) {
    if (c->f32.u[0]) return RBGS_OK;
    c->f32.n = c->g.n;
    c->f32.W = colour_width_bytes(c->g.n, 4);
    const size_t bytes = (size_t)c->g.rows * c->f32.W * sizeof(float);
    for (int q = 0; q < 2; ++q) {
        rbgs_status st;
        if ((st = alloc_zero(reinterpret_cast<void **>(&c->f32.u[q]), bytes, c->stream)) != RBGS_OK) return st;
        if ((st = alloc_zero(reinterpret_cast<void **>(&c->f32.hf[q]), bytes, c->stream)) != RBGS_OK) return st;
        if ((c->kernel32 == RBGS_KERNEL_TEMPORAL || c->kernel32 == RBGS_KERNEL_WAVEFRONT) &&
            (st = alloc_zero(reinterpret_cast<void **>(&c->f32.alt[q]), bytes, c->stream)) != RBGS_OK)
            return st;
    }
    c->f32.maps_ready = false;
    return RBGS_OK;
}

// A bounded device-side wait gave up in an earlier launch?  (Reads after a stream sync.)
rbgs_status check_device_status(rbgs_ctx *c) {
    RBGS_CUDA(cudaMemcpyAsync(c->hstatus, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    RBGS_CUDA(cudaStreamSynchronize(c->stream));
    if (*c->hstatus) {
        set_error("a bounded device-side wait timed out (status %d)", *c->hstatus);
        return RBGS_ETIMEOUT;
    }
    return RBGS_OK;
}

rbgs_status enqueue_sweeps(rbgs_ctx *c, long nsweeps, cudaStream_t s) {
    if (c->fused) {
        for (long it = 0; it < nsweeps; ++it) {
            rbgs_status st = launch_fused_half_sweep(c, 0, s);
            if (st == RBGS_OK) st = launch_fused_half_sweep(c, 1, s);
            if (st != RBGS_OK) return st;
        }
        return RBGS_OK;
    }
    if (c->kernel == RBGS_KERNEL_TEMPORAL) return launch_temporal_sweeps(c, nsweeps, s);
    if (c->kernel == RBGS_KERNEL_WAVEFRONT) {
        const long passes = nsweeps / c->tblock_k;
        for (long q = 0; q < passes; ++q) {
            rbgs_status st = launch_wavefront_pass<double>(c->f64, c->tblock_k, s);
            if (st != RBGS_OK) return st;
        }
        nsweeps -= passes * c->tblock_k;
    }
    return launch_sweeps_f64(c, nsweeps, s);
}

rbgs_status ensure_graph(rbgs_ctx *c) {
    if (c->graph) return RBGS_OK;
    cudaGraph_t graph = nullptr;
    RBGS_CUDA(cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal));
    rbgs_status st = enqueue_sweeps(c, kGraphSweeps, c->capture);
    cudaError_t e = cudaStreamEndCapture(c->capture, &graph);
    if (st != RBGS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) {
        set_error("graph capture failed: %s", cudaGetErrorString(e));
        return RBGS_ECUDA;
    }
    e = cudaGraphInstantiate(&c->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        c->graph = nullptr;
        set_error("graph instantiation failed: %s", cudaGetErrorString(e));
        return RBGS_ECUDA;
    }
    c->graph_sweeps = kGraphSweeps;
    return RBGS_OK;
}

// nsweeps FP64 sweeps: one cooperative launch, cached graphs of kGraphSweeps sweeps on small
// grids, or direct / temporally blocked launches.
rbgs_status sweeps_f64(rbgs_ctx *c, long nsweeps) {
    if (c->fused) {
        // blocks of at most kFusedChunk sweeps, each at the scale chosen when it starts; the
        // sweeps of a block as cached graphs of kGraphSweeps sweeps at every size (the
        // half-sweeps are short even on large grids, so the launch gaps still count)
        while (nsweeps > 0) {
            long m = nsweeps < kFusedChunk ? nsweeps : kFusedChunk;
            nsweeps -= m;
            rbgs_status st = launch_fused_prepare(c, m, c->stream);
            if (st != RBGS_OK) return st;
            if (m >= kGraphSweeps) {
                if ((st = ensure_graph(c)) != RBGS_OK) return st;
                while (m >= c->graph_sweeps) {
                    RBGS_CUDA(cudaGraphLaunch(c->graph, c->stream));
                    m -= c->graph_sweeps;
                }
            }
            if ((st = enqueue_sweeps(c, m, c->stream)) != RBGS_OK) return st;
        }
        return RBGS_OK;
    }
    if (use_persistent(c)) return launch_persistent_sweeps<double>(c->f64, nsweeps, c->pcounter, c->dstatus, c->stream);
    if (c->kernel == RBGS_KERNEL_COLOUR && c->g.n <= kGraphMaxN && nsweeps >= kGraphSweeps) {
        rbgs_status st = ensure_graph(c);
        if (st != RBGS_OK) return st;
        while (nsweeps >= c->graph_sweeps) {
            RBGS_CUDA(cudaGraphLaunch(c->graph, c->stream));
            nsweeps -= c->graph_sweeps;
        }
    }
    return enqueue_sweeps(c, nsweeps, c->stream);
}

// rho and max |rt| of the current FP64 iterate (synchronises the stream).
rbgs_status defect_stats(rbgs_ctx *c, double *rho, double *mx) {
    rbgs_status st = launch_defect(c, false, 1.0, c->stream);
    if (st != RBGS_OK) return st;
    RBGS_CUDA(cudaMemcpyAsync(c->hsum, c->dsum, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if ((st = check_device_status(c)) != RBGS_OK) return st;
    const double r2 = c->hsum[0];
    *mx = c->hsum[2];
    *rho = c->den2 > 0.0 ? std::sqrt(r2) / std::sqrt(c->den2) : std::sqrt(r2);
    if (!std::isfinite(*rho)) {
        set_error("residual is not finite");
        return RBGS_ENONFINITE;
    }
    return RBGS_OK;
}

rbgs_status inner_sweeps_f32(rbgs_ctx *c, long m) {
    // small grids: all m sweeps in one launch of one thread-block cluster
    if (c->kernel32 == RBGS_KERNEL_COLOUR && c->opts.tile_rows == 0 && c->g.n <= kClusterMaxN &&
        cluster_sweeps_f32_fit(c->g.n, c->f32.W))
        return launch_cluster_sweeps_f32(c->f32, m, c->stream);
    // full inner blocks of one-launch-per-colour sweeps on small grids: a cached graph
    if (c->kernel32 == RBGS_KERNEL_COLOUR && m == c->inner_sweeps && c->g.n <= kGraphMaxN) {
        if (!c->graph32) {
            cudaGraph_t graph = nullptr;
            RBGS_CUDA(cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal));
            rbgs_status st = launch_sweeps_f32(c->f32, m, c->capture);
            cudaError_t e = cudaStreamEndCapture(c->capture, &graph);
            if (st != RBGS_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if (e != cudaSuccess) {
                set_error("graph capture failed: %s", cudaGetErrorString(e));
                return RBGS_ECUDA;
            }
            e = cudaGraphInstantiate(&c->graph32, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                c->graph32 = nullptr;
                set_error("graph instantiation failed: %s", cudaGetErrorString(e));
                return RBGS_ECUDA;
            }
        }
        RBGS_CUDA(cudaGraphLaunch(c->graph32, c->stream));
        return RBGS_OK;
    }
    if (c->kernel32 == RBGS_KERNEL_TEMPORAL || c->kernel32 == RBGS_KERNEL_WAVEFRONT) {
        const int k = c->tblock_k32;
        const long passes = m / k;
        for (long q = 0; q < passes; ++q) {
            rbgs_status st = c->kernel32 == RBGS_KERNEL_TEMPORAL
                                 ? launch_temporal_pass<float>(c->f32, k, c->dstatus, c->stream)
                                 : launch_wavefront_pass<float>(c->f32, k, c->stream);
            if (st != RBGS_OK) return st;
        }
        m -= passes * k;
    }
    return launch_sweeps_f32(c->f32, m, c->stream);
}

// Mixed-precision iterative refinement: FP64 defect and correction, FP32 sweeps.
rbgs_status refine_solve(rbgs_ctx *c, double tol, long *done_out, double *rho_out) {
    c->black_fresh = false;  // the corrections move every point
    rbgs_status st = ensure_f32(c);
    long done = 0;
    double rho = 0.0, mx = 0.0;
    if (st == RBGS_OK) st = defect_stats(c, &rho, &mx);
    while (st == RBGS_OK && !(rho <= tol) && done < c->opts.max_sweeps) {
        int e = 0;
        std::frexp(mx, &e);  // mx = m 2^e, m in [0.5, 1)
        const double down = std::ldexp(1.0, -e), up = std::ldexp(1.0, e);
        if ((st = launch_defect(c, true, down, c->stream)) != RBGS_OK) break;
        const size_t bytes = (size_t)c->g.rows * c->f32.W * sizeof(float);
        for (int q = 0; q < 2; ++q) {
            if (cudaMemsetAsync(c->f32.u[q], 0, bytes, c->stream) != cudaSuccess) {
                cudaGetLastError();
                set_error("cudaMemsetAsync failed");
                st = RBGS_ECUDA;
            }
        }
        if (st != RBGS_OK) break;
        long m = c->inner_sweeps;
        if (m > c->opts.max_sweeps - done) m = c->opts.max_sweeps - done;
        if ((st = inner_sweeps_f32(c, m)) != RBGS_OK) break;
        if ((st = launch_correct(c, up, c->stream)) != RBGS_OK) break;
        done += m;
        st = defect_stats(c, &rho, &mx);
    }
    if (done_out) *done_out = done;
    if (rho_out) *rho_out = rho;
    if (st == RBGS_OK && !(rho <= tol)) {
        set_error("not converged after %ld sweeps (rho = %.3e)", done, rho);
        st = RBGS_ENOTCONV;
    }
    return st;
}

// Buffers, copy streams and events of rbgs_run_stream (allocated on first use; staging
// only for the directions that see host memory).
rbgs_status ensure_stream(rbgs_ctx *c, bool in_host, bool out_host, int count) {
    const size_t nat_f = (size_t)c->g.n * c->g.n * sizeof(double);
    const size_t nat_u = (size_t)c->g.rows * c->g.rows * sizeof(double);
    bool ok = true;
    for (int q = 0; q < 2 && ok; ++q) {
        if (in_host && !c->sin_f[q])
            ok = cudaMalloc(&c->sin_f[q], nat_f) == cudaSuccess && cudaMalloc(&c->sin_u[q], nat_u) == cudaSuccess;
        if (ok && out_host && !c->sout[q]) ok = cudaMalloc(&c->sout[q], nat_u) == cudaSuccess;
        if (ok && !c->ev_copied[q])
            ok = cudaEventCreateWithFlags(&c->ev_copied[q], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&c->ev_packed[q], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&c->ev_unpacked[q], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&c->ev_out[q], cudaEventDisableTiming) == cudaSuccess;
    }
    if (ok && !c->h2d)
        ok = cudaStreamCreateWithFlags(&c->h2d, cudaStreamNonBlocking) == cudaSuccess &&
             cudaStreamCreateWithFlags(&c->d2h, cudaStreamNonBlocking) == cudaSuccess;
    if (ok && (size_t)count > c->res_cap) {
        cudaFree(c->dres);
        if (c->hres) cudaFreeHost(c->hres);
        c->dres = nullptr;
        c->hres = nullptr;
        c->res_cap = 0;
        ok = cudaMalloc(&c->dres, 2 * (size_t)count * sizeof(double)) == cudaSuccess &&
             cudaMallocHost(&c->hres, 2 * (size_t)count * sizeof(double)) == cudaSuccess;
        if (ok) c->res_cap = (size_t)count;
    }
    if (!ok) {
        cudaGetLastError();
        set_error("rbgs_run_stream: allocation of staging buffers, streams or events failed");
        return RBGS_ENOMEM;
    }
    return RBGS_OK;
}

}  // namespace
}  // namespace rbgs

using namespace rbgs;

extern "C" {

void rbgs_default_opts(rbgs_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = RBGS_FP64;
    o->kernel = RBGS_KERNEL_AUTO;
    o->check_every = 100;
    o->max_sweeps = 1000000000L;
    o->fp64_emulate = -1;
    o->fma = 0;
    o->stall_checks = 0;
    o->max_seconds = 0.0;
}

const char *rbgs_last_error(void) { return g_err; }

rbgs_status rbgs_create(int n, double h2, const double *f, const double *u_init,
                        const rbgs_opts *opts, void *cuda_stream, rbgs_t *out) {
    clear_error();
    if (!out) { set_error("out is NULL"); return RBGS_EINVAL; }
    *out = nullptr;
    if (n < 1 || n > kMaxN) { set_error("n = %d outside 1..%d", n, kMaxN); return RBGS_EINVAL; }
    if (!(h2 > 0.0) || !std::isfinite(h2)) { set_error("h2 must be finite and > 0"); return RBGS_EINVAL; }
    if (!f || !u_init) { set_error("f and u_init must not be NULL"); return RBGS_EINVAL; }
    rbgs_opts o;
    rbgs_default_opts(&o);
    if (opts) o = *opts;
    if (o.check_every <= 0) o.check_every = 100;
    if (o.max_sweeps <= 0) o.max_sweeps = 1000000000L;
    if (o.precision != RBGS_FP64 && o.precision != RBGS_FP32_REFINE) {
        set_error("unknown precision %d", o.precision); return RBGS_EINVAL;
    }
    if (o.kernel < RBGS_KERNEL_AUTO || o.kernel > RBGS_KERNEL_PERSISTENT) {
        set_error("unknown kernel %d", o.kernel); return RBGS_EINVAL;
    }
    if (o.kernel == RBGS_KERNEL_PERSISTENT && n > kPersistMaxN) {
        set_error("RBGS_KERNEL_PERSISTENT supports n <= %d", kPersistMaxN); return RBGS_EINVAL;
    }
    if (o.fp64_emulate != -1 && !emulation_split_supported(o.fp64_emulate)) {
        set_error("unsupported fp64_emulate %d", o.fp64_emulate); return RBGS_EINVAL;
    }
    if (o.sweep_values != 0 && o.sweep_values != 2 && o.sweep_values != 4) {
        set_error("sweep_values must be 0, 2 or 4"); return RBGS_EINVAL;
    }
    if (o.int_rows < -1) {
        set_error("int_rows must be >= -1"); return RBGS_EINVAL;
    }
    if (o.sweep_rows != 0 && o.sweep_rows != 1 && o.sweep_rows != 2) {
        set_error("sweep_rows must be 0, 1 or 2"); return RBGS_EINVAL;
    }
    if (o.fma != 0 && o.fma != 1) {
        set_error("fma must be 0 (bit-exact) or 1 (fused)"); return RBGS_EINVAL;
    }
    if (o.fma == 1 && o.precision != RBGS_FP64) {
        set_error("fma = 1 applies to RBGS_FP64 sweeps only"); return RBGS_EINVAL;
    }
    if (o.fma == 1 && o.kernel != RBGS_KERNEL_AUTO && o.kernel != RBGS_KERNEL_COLOUR) {
        set_error("fma = 1 runs one launch per colour (kernel AUTO or COLOUR)"); return RBGS_EINVAL;
    }
    if (o.stall_checks < -1) {
        set_error("stall_checks must be >= -1"); return RBGS_EINVAL;
    }
    if (!(o.max_seconds >= 0.0) || !std::isfinite(o.max_seconds)) {
        set_error("max_seconds must be finite and >= 0"); return RBGS_EINVAL;
    }
    if (o.tile_rows < 0 || o.tblock_k < 0 || o.inner_sweeps < 0) {
        set_error("negative tile_rows / tblock_k / inner_sweeps"); return RBGS_EINVAL;
    }
    if (o.kernel == RBGS_KERNEL_WAVEFRONT) {
        if (o.tblock_k && o.precision == RBGS_FP64 && o.tblock_k != 2 && o.tblock_k != 4) {
            set_error("tblock_k of the FP64 wavefront must be 2 or 4"); return RBGS_EINVAL;
        }
        if (o.tblock_k && o.precision == RBGS_FP32_REFINE && o.tblock_k != 2 && o.tblock_k != 4 &&
            o.tblock_k != 6) {
            set_error("tblock_k of the FP32 wavefront must be 2, 4 or 6"); return RBGS_EINVAL;
        }
    } else {
        if (o.tblock_k && o.precision == RBGS_FP64 && o.tblock_k != 1 && o.tblock_k != 2 && o.tblock_k != 4) {
            set_error("tblock_k for FP64 sweeps must be 1, 2 or 4"); return RBGS_EINVAL;
        }
        if (o.tblock_k && o.precision == RBGS_FP32_REFINE && o.tblock_k != 2 && o.tblock_k != 4 &&
            o.tblock_k != 8) {
            set_error("tblock_k for FP32 inner sweeps must be 2, 4 or 8"); return RBGS_EINVAL;
        }
    }

    rbgs_ctx *c = new (std::nothrow) rbgs_ctx();
    if (!c) { set_error("out of host memory"); return RBGS_ENOMEM; }
    c->g = make_geometry(n);
    c->h2 = h2;
    c->opts = o;
    c->stream = (cudaStream_t)cuda_stream;
    // automatic kernels (measured on GB300): FP64 sweeps run in one cooperative launch from
    // 416^2 to 32768^2 with the default launch shape (1.15x at 511^2 to 1.53x at 2047^2 and
    // 1.10x at 16383^2 over one launch per colour), else one launch per colour with cached
    // graphs (the register wavefront reaches the same FP64-pipe limit, with overlap work on
    // top); the FP32 inner sweeps of the refinement run the register wavefront above 2048^2
    // (1.6x) and one launch per colour (with graphs) on smaller grids
    const bool auto_k = o.kernel == RBGS_KERNEL_AUTO && o.tblock_k == 0;
    const bool default_shape = o.fp64_emulate == -1 && o.int_rows <= 0 && (o.sweep_values == 0 || o.sweep_values == 2) &&
                               (o.sweep_rows == 0 || o.sweep_rows == 1) && o.tile_rows == 0;
    c->fused = o.fma == 1;
    c->kernel = c->fused ? RBGS_KERNEL_COLOUR
                : o.kernel != RBGS_KERNEL_AUTO ? o.kernel
                : (default_shape && n >= kPersistMinN && n <= kPersistMaxN) ? RBGS_KERNEL_PERSISTENT
                                                                            : RBGS_KERNEL_COLOUR;
    c->emulate = o.fp64_emulate == -1 ? 0x00 : o.fp64_emulate;
    c->pts = o.sweep_values ? o.sweep_values : (c->fused ? 4 : 2);
    if (o.tile_rows) {
        c->tile_rows = o.tile_rows;
    } else {
        // strips of up to 16 rows, fewer when that leaves fewer than ~4 blocks per SM (16
        // measured 0.6% faster than 32 at 16384^2, 64 slower)
        int sms = 0;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            sms = 152;
        }
        const long gx = (active_width(n) + c->pts * kSweepThreads - 1) / (c->pts * kSweepThreads);
        long r = (long)n * gx / (4L * sms);
        c->tile_rows = (int)(r < 1 ? 1 : (r > 16 ? 16 : r));
    }
    if (c->tile_rows < (n + 65534) / 65535) c->tile_rows = (n + 65534) / 65535;  // grid.y limit
    c->sweep_rows = o.sweep_rows ? o.sweep_rows : 1;
    c->int_rows = o.int_rows > 0 ? o.int_rows : 0;
    // FP64 sweeps: temporal depth (used when kernel == TEMPORAL)
    c->tblock_k = (o.precision == RBGS_FP64 && o.tblock_k) ? o.tblock_k : 2;
    // FP32 inner sweeps of the refinement (the TMA-tiled temporal kernel measured slower
    // than one launch per colour on GB300; the register wavefront faster above 2048^2)
    c->kernel32 = o.kernel == RBGS_KERNEL_AUTO ? ((auto_k && n > 2048) ? RBGS_KERNEL_WAVEFRONT
                                                                       : RBGS_KERNEL_COLOUR)
                  : o.kernel == RBGS_KERNEL_PERSISTENT ? RBGS_KERNEL_COLOUR
                                                        : o.kernel;
    c->tblock_k32 = (o.precision == RBGS_FP32_REFINE && o.tblock_k) ? o.tblock_k : 4;
    c->inner_sweeps = o.inner_sweeps ? o.inner_sweeps : 100;
    c->f64.n = n;
    c->f64.W = c->g.W;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        set_error("no CUDA device");
        return RBGS_ECUDA;
    }
    const size_t bytes = c->g.colour_elems() * sizeof(double);
    bool ok = true;
    for (int q = 0; q < 2 && ok; ++q) {
        ok = cudaMalloc(&c->f64.u[q], bytes) == cudaSuccess && cudaMalloc(&c->f64.hf[q], bytes) == cudaSuccess;
    }
    ok = ok && cudaMalloc(&c->partials, 2 * kMaxPartials * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc(&c->dsum, 4 * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc(&c->dstatus, sizeof(int)) == cudaSuccess;
    ok = ok && cudaMalloc(&c->pcounter, sizeof(unsigned)) == cudaSuccess;
    ok = ok && cudaMallocHost(&c->hsum, 4 * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMallocHost(&c->hstatus, sizeof(int)) == cudaSuccess;
    for (int q = 0; q < 2 && ok && c->fused; ++q) ok = cudaMalloc(&c->hq[q], c->g.colour_elems() * sizeof(int64_t)) == cudaSuccess;
    ok = ok && (!c->fused || cudaMalloc(&c->fwords, 3 * sizeof(unsigned long long)) == cudaSuccess);
    ok = ok && cudaMemsetAsync(c->dstatus, 0, sizeof(int), c->stream) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_ctx(c);
        set_error("allocation of %zu bytes of solver state failed", 4 * bytes);
        return RBGS_ENOMEM;
    }
    if (cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        free_ctx(c);
        set_error("stream creation failed");
        return RBGS_ECUDA;
    }
    rbgs_status st = RBGS_OK;
    if (c->kernel == RBGS_KERNEL_TEMPORAL || c->kernel == RBGS_KERNEL_WAVEFRONT) st = ensure_f64_alt(c);
    if (st == RBGS_OK) st = load_problem(c, f, u_init);
    if (st != RBGS_OK) {
        free_ctx(c);
        return st;
    }
    *out = c;
    return RBGS_OK;
}

rbgs_status rbgs_sweep(rbgs_t c, long nsweeps) {
    clear_error();
    if (!c) { set_error("ctx is NULL"); return RBGS_EINVAL; }
    if (nsweeps < 0) { set_error("nsweeps < 0"); return RBGS_EINVAL; }
    if (nsweeps == 0) return RBGS_OK;
    const rbgs_status st = sweeps_f64(c, nsweeps);
    // after a completed bit-exact sweep the black points' residual is exactly zero
    // (residual.cu); the fused update rounds the black points differently
    c->black_fresh = st == RBGS_OK && !c->fused;
    return st;
}

rbgs_status rbgs_residual(rbgs_t c, double *rel) {
    clear_error();
    if (!c || !rel) { set_error("ctx and rel must not be NULL"); return RBGS_EINVAL; }
    rbgs_status st = launch_residual_sum(c, c->stream);
    if (st != RBGS_OK) return st;
    RBGS_CUDA(cudaMemcpyAsync(c->hsum, c->dsum, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if ((st = check_device_status(c)) != RBGS_OK) return st;
    const double r2 = c->hsum[0];
    *rel = c->den2 > 0.0 ? std::sqrt(r2) / std::sqrt(c->den2) : std::sqrt(r2);
    if (!std::isfinite(*rel)) {
        set_error("residual is not finite");
        return RBGS_ENONFINITE;
    }
    return RBGS_OK;
}

rbgs_status rbgs_solve(rbgs_t c, double tol, long *sweeps_done, double *rel) {
    clear_error();
    if (!c) { set_error("ctx is NULL"); return RBGS_EINVAL; }
    if (!(tol >= 0.0)) { set_error("tol must be >= 0"); return RBGS_EINVAL; }
    if (c->opts.precision == RBGS_FP32_REFINE) return refine_solve(c, tol, sweeps_done, rel);
    long done = 0;
    double rho = 0.0;
    rbgs_status st = rbgs_residual(c, &rho);
    const int stall_limit = c->opts.stall_checks == 0 ? kDefaultStallChecks : c->opts.stall_checks;
    double best = rho;
    int since_best = 0;
    bool stalled = false;
    while (st == RBGS_OK && !(rho <= tol) && done < c->opts.max_sweeps) {
        long k = c->opts.check_every;
        if (k > c->opts.max_sweeps - done) k = c->opts.max_sweeps - done;
        if ((st = rbgs_sweep(c, k)) != RBGS_OK) break;
        done += k;
        if ((st = rbgs_residual(c, &rho)) != RBGS_OK) break;
        if (rho < best) {
            best = rho;
            since_best = 0;
        } else if (stall_limit > 0 && ++since_best >= stall_limit) {
            stalled = true;
            break;
        }
    }
    if (sweeps_done) *sweeps_done = done;
    if (rel) *rel = rho;
    if (st == RBGS_OK && !(rho <= tol)) {
        if (stalled)
            set_error("stalled: rho = %.3e has not gone below its minimum %.3e for %d checks (%ld sweeps)", rho,
                      best, stall_limit, done);
        else
            set_error("not converged after %ld sweeps (rho = %.3e)", done, rho);
        st = RBGS_ENOTCONV;
    }
    return st;
}

rbgs_status rbgs_get_solution(rbgs_t c, double *u_out) {
    clear_error();
    if (!c || !u_out) { set_error("ctx and u_out must not be NULL"); return RBGS_EINVAL; }
    const size_t count = (size_t)c->g.rows * c->g.rows;
    if (device_accessible(u_out)) {
        return launch_unpack_u(c->g, c->f64.u[0], c->f64.u[1], u_out, c->stream);
    }
    if (!c->staging) {
        if (cudaMalloc(&c->staging, count * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            set_error("staging allocation failed");
            return RBGS_ENOMEM;
        }
    }
    rbgs_status st = launch_unpack_u(c->g, c->f64.u[0], c->f64.u[1], c->staging, c->stream);
    if (st != RBGS_OK) return st;
    RBGS_CUDA(cudaMemcpyAsync(u_out, c->staging, count * sizeof(double), cudaMemcpyDefault, c->stream));
    RBGS_CUDA(cudaStreamSynchronize(c->stream));
    return RBGS_OK;
}

rbgs_status rbgs_set_solution(rbgs_t c, const double *u_in) {
    clear_error();
    if (!c || !u_in) { set_error("ctx and u_in must not be NULL"); return RBGS_EINVAL; }
    return load_problem(c, nullptr, u_in);
}

rbgs_status rbgs_set_problem(rbgs_t c, const double *f, const double *u_init) {
    clear_error();
    if (!c || !f || !u_init) { set_error("ctx, f and u_init must not be NULL"); return RBGS_EINVAL; }
    return load_problem(c, f, u_init);
}

rbgs_status rbgs_run_stream(rbgs_t c, int count, const double *const *f, const double *const *u_init, long nsweeps,
                            double *const *u_out, double *rho) {
    clear_error();
    if (!c || count < 0 || nsweeps < 0 || (count > 0 && (!f || !u_init || !u_out))) {
        set_error("rbgs_run_stream: ctx, f, u_init and u_out must be given, count and nsweeps >= 0");
        return RBGS_EINVAL;
    }
    for (int q = 0; q < count; ++q) {
        if (!f[q] || !u_init[q] || !u_out[q]) {
            set_error("rbgs_run_stream: problem %d has a NULL pointer", q);
            return RBGS_EINVAL;
        }
    }
    if (count == 0) return RBGS_OK;
    if (c->opts.precision != RBGS_FP64) {
        set_error("rbgs_run_stream runs RBGS_FP64 sweeps (fused or bit-exact)");
        return RBGS_EINVAL;
    }
    const Geometry &g = c->g;
    const size_t bytes_f = (size_t)g.n * g.n * sizeof(double), bytes_u = (size_t)g.rows * g.rows * sizeof(double);
    std::vector<char> in_dev(count), out_dev(count);
    bool any_in_host = false, any_out_host = false;
    for (int q = 0; q < count; ++q) {
        in_dev[q] = device_accessible(f[q]) && device_accessible(u_init[q]);
        out_dev[q] = device_accessible(u_out[q]);
        any_in_host |= !in_dev[q];
        any_out_host |= !out_dev[q];
    }
    rbgs_status st = ensure_stream(c, any_in_host, any_out_host, count);
    if (st != RBGS_OK) return st;
    cudaStream_t ms = c->stream;
    // host -> device copy of problem q's inputs into staging buffer q % 2, once the pack of
    // problem q - 2 (the buffer's previous reader) has run
    auto copy_in = [&](int q) -> rbgs_status {
        if (in_dev[q]) return RBGS_OK;
        const int b = q & 1;
        if (q >= 2) RBGS_CUDA(cudaStreamWaitEvent(c->h2d, c->ev_packed[b], 0));
        RBGS_CUDA(cudaMemcpyAsync(c->sin_f[b], f[q], bytes_f, cudaMemcpyDefault, c->h2d));
        RBGS_CUDA(cudaMemcpyAsync(c->sin_u[b], u_init[q], bytes_u, cudaMemcpyDefault, c->h2d));
        RBGS_CUDA(cudaEventRecord(c->ev_copied[b], c->h2d));
        return RBGS_OK;
    };
    // the caller's earlier work on the context's stream comes first
    RBGS_CUDA(cudaEventRecord(c->ev_unpacked[1], ms));
    RBGS_CUDA(cudaStreamWaitEvent(c->h2d, c->ev_unpacked[1], 0));
    RBGS_CUDA(cudaStreamWaitEvent(c->d2h, c->ev_unpacked[1], 0));
    if ((st = copy_in(0)) != RBGS_OK) return st;
    for (int q = 0; q < count; ++q) {
        const int b = q & 1;
        const double *fv = f[q], *uv = u_init[q];
        if (!in_dev[q]) {
            RBGS_CUDA(cudaStreamWaitEvent(ms, c->ev_copied[b], 0));
            fv = c->sin_f[b];
            uv = c->sin_u[b];
        }
        if ((st = enqueue_pack(c, fv, uv)) != RBGS_OK) return st;
        RBGS_CUDA(cudaEventRecord(c->ev_packed[b], ms));
        RBGS_CUDA(cudaMemcpyAsync(c->dres + 2 * q, c->dsum + 1, sizeof(double), cudaMemcpyDeviceToDevice, ms));
        // the next problem's inputs move while this one sweeps
        if (q + 1 < count && (st = copy_in(q + 1)) != RBGS_OK) return st;
        if (nsweeps > 0) {
            if ((st = sweeps_f64(c, nsweeps)) != RBGS_OK) return st;
            c->black_fresh = !c->fused;
        }
        if ((st = launch_residual_sum(c, ms)) != RBGS_OK) return st;
        RBGS_CUDA(cudaMemcpyAsync(c->dres + 2 * q + 1, c->dsum, sizeof(double), cudaMemcpyDeviceToDevice, ms));
        if (out_dev[q]) {
            if ((st = launch_unpack_u(g, c->f64.u[0], c->f64.u[1], u_out[q], ms)) != RBGS_OK) return st;
        } else {
            // staging buffer b is free once the copy-out of problem q - 2 has finished; this
            // solution then leaves while the next problem sweeps
            if (q >= 2) RBGS_CUDA(cudaStreamWaitEvent(ms, c->ev_out[b], 0));
            if ((st = launch_unpack_u(g, c->f64.u[0], c->f64.u[1], c->sout[b], ms)) != RBGS_OK) return st;
            RBGS_CUDA(cudaEventRecord(c->ev_unpacked[b], ms));
            RBGS_CUDA(cudaStreamWaitEvent(c->d2h, c->ev_unpacked[b], 0));
            RBGS_CUDA(cudaMemcpyAsync(u_out[q], c->sout[b], bytes_u, cudaMemcpyDefault, c->d2h));
            RBGS_CUDA(cudaEventRecord(c->ev_out[b], c->d2h));
        }
    }
    RBGS_CUDA(cudaMemcpyAsync(c->hres, c->dres, 2 * (size_t)count * sizeof(double), cudaMemcpyDeviceToHost, ms));
    // later work on the context's stream (and events the caller records there) follows the
    // last copies
    RBGS_CUDA(cudaEventRecord(c->ev_copied[0], c->h2d));
    RBGS_CUDA(cudaEventRecord(c->ev_out[0], c->d2h));
    RBGS_CUDA(cudaStreamWaitEvent(ms, c->ev_copied[0], 0));
    RBGS_CUDA(cudaStreamWaitEvent(ms, c->ev_out[0], 0));
    if ((st = check_device_status(c)) != RBGS_OK) return st;
    rbgs_status result = RBGS_OK;
    for (int q = 0; q < count; ++q) {
        const double den2 = c->hres[2 * q], r2 = c->hres[2 * q + 1];
        const double r = den2 > 0.0 ? std::sqrt(r2) / std::sqrt(den2) : std::sqrt(r2);
        if (rho) rho[q] = r;
        if (!std::isfinite(r) && result == RBGS_OK) {
            set_error("rbgs_run_stream: problem %d: residual is not finite", q);
            result = RBGS_ENONFINITE;
        }
    }
    c->den2 = c->hres[2 * (count - 1)];
    return result;
}

void rbgs_destroy(rbgs_t c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
}

}  // extern "C"
