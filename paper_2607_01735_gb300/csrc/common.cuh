// Shared definitions of librbgs: the solver context, the colour-split layout and error
// plumbing.  Internal to the library (the public ABI is include/rbgs.h).
//
// Colour-split layout (the red/black split storage of Section 2.1 of the paper, with
// padded rows): colour c (0 red, 1 black) of grid row i, 0 <= i <= N+1, is a row of W
// values; element k holds the natural point j = 2k + ((i + c) & 1).  A red point and its
// north/south neighbours share k; its west/east neighbours sit at k-1/k when the row's
// red offset (i & 1) is 0 and at k/k+1 when it is 1.  W = ceil((N+2)/2) rounded up to a
// multiple of 32 values (256 bytes), so every row starts on a 256-byte boundary and a
// half-sweep reads and writes each value of a colour once.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/rbgs.h"
#include "field.cuh"

namespace rbgs {

// message for rbgs_last_error(); thread-local
void set_error(const char *fmt, ...);
void clear_error();

#define RBGS_CUDA(call)                                                                  \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            ::rbgs::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                              __FILE__, __LINE__);                                       \
            return RBGS_ECUDA;                                                           \
        }                                                                                \
    } while (0)

#define RBGS_LAUNCH_CHECK()                                                              \
    do {                                                                                 \
        cudaError_t e_ = cudaGetLastError();                                             \
        if (e_ != cudaSuccess) {                                                         \
            ::rbgs::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_), \
                              __FILE__, __LINE__);                                       \
            return RBGS_ECUDA;                                                           \
        }                                                                                \
    } while (0)

constexpr int kRowAlign = 32;  // values per row alignment unit (256 B of FP64)

inline int colour_width(int n) {
    int w = (n + 3) / 2;
    return (w + kRowAlign - 1) / kRowAlign * kRowAlign;
}

// Geometry of one grid in the colour-split layout.
struct Geometry {
    int n;       // interior points per side
    int W;       // values per colour row (padded)
    int rows;    // n + 2
    size_t colour_elems() const { return (size_t)rows * (size_t)W; }
};

inline Geometry make_geometry(int n) { return Geometry{n, colour_width(n), n + 2}; }

// Residual reduction scratch: one partial sum per thread block.
constexpr int kMaxPartials = 8192;

struct Ctx;

}  // namespace rbgs

struct rbgs_ctx {
    rbgs::Geometry g;
    double h2;
    rbgs_opts opts;
    cudaStream_t stream;        // caller's stream (may be 0)
    cudaStream_t capture;       // private stream used only to capture graphs
    int device;
    // FP64 iterate, its temporal partner and the scaled right-hand side h2*f, colour-split
    rbgs::ColourField<double> f64;
    // FP32 correction (u), its partner (alt) and scaled defect (hf) of the mixed-precision
    // refinement (allocated on first use)
    rbgs::ColourField<float> f32;
    int *dstatus;               // device: nonzero after a bounded wait gave up
    // natural-layout staging for host I/O (allocated on demand)
    double *staging;
    // reduction scratch and results
    double *partials;
    double *dsum;               // device: [0] sum r^2, [1] sum b^2, [2] max |r|
    double *hsum;               // pinned host mirror
    double den2;                // sum (h^2 b)^2, fixed by f and the ring
    // cached graph of `graph_sweeps` sweeps
    cudaGraphExec_t graph;
    long graph_sweeps;
    cudaGraphExec_t graph32;    // cached graph of inner_sweeps FP32 sweeps (refinement)
    int kernel;                 // resolved rbgs_kernel
    int emulate;                // resolved FP64 emulation split
    int tile_rows;              // resolved rows per block
    int pts;                    // values per thread in the half-sweep (2 or 4)
    int sweep_rows;             // rows per loop step in the half-sweep (1 or 2)
    int int_rows;               // hybrid FP64 half-sweep: integer-pipe rows per strip pair (0: off)
    int tblock_k;               // resolved temporal depth (FP64)
    int tblock_k32;             // resolved temporal depth (FP32 inner sweeps)
    int inner_sweeps;           // resolved FP32 sweeps per correction
    int kernel32;               // resolved inner kernel for the FP32 sweeps
    int *hstatus;               // pinned host mirror of dstatus
    unsigned *pcounter;         // device: grid-barrier counter of the cooperative sweep launch
    bool black_fresh;           // the FP64 iterate is the result of a full sweep (black rt == 0)
    // fused FP64 update (opts.fma = 1): h2 f on the fixed-point grid of the current block of
    // sweeps, per colour, and [0] max |u| bits, [1] max |h2 f| bits, [2] the block's scale e
    bool fused;
    int64_t *hq[2];
    unsigned long long *fwords;
    // rbgs_run_stream: double-buffered natural-layout device staging of the inputs (f, u) and
    // of the solution, one copy stream per direction, their events, and per-problem sums
    double *sin_f[2], *sin_u[2], *sout[2];
    cudaStream_t h2d, d2h;
    cudaEvent_t ev_copied[2], ev_packed[2], ev_unpacked[2], ev_out[2];
    double *dres, *hres;        // device / pinned host: [2q] sum (h^2 b)^2, [2q+1] sum rt^2
    size_t res_cap;             // problems dres and hres hold
};

namespace rbgs {

// launchers implemented in the .cu files; all enqueue on `s` and return a status
rbgs_status launch_pack_u(const Geometry &g, const double *u_nat, double *red, double *black,
                          cudaStream_t s);
rbgs_status launch_pack_f(const Geometry &g, double h2, const double *f_nat, double *hf_red,
                          double *hf_black, cudaStream_t s);
rbgs_status launch_unpack_u(const Geometry &g, const double *red, const double *black,
                            double *u_nat, cudaStream_t s);
rbgs_status launch_half_sweep(const rbgs_ctx *c, int colour, cudaStream_t s);
rbgs_status launch_sweeps_f64(const rbgs_ctx *c, long nsweeps, cudaStream_t s);
rbgs_status launch_residual_sum(const rbgs_ctx *c, cudaStream_t s);   // -> dsum[0]
rbgs_status launch_rhs_norm(const rbgs_ctx *c, cudaStream_t s);       // -> dsum[1]
rbgs_status launch_temporal_sweeps(rbgs_ctx *c, long nsweeps, cudaStream_t s);
template <typename T>
rbgs_status launch_temporal_pass(ColourField<T> &fld, int k, int *status, cudaStream_t s);
rbgs_status launch_sweeps_f32(const ColourField<float> &fld, long nsweeps, cudaStream_t s);
// one register-wavefront pass of k sweeps from fld.u into fld.alt, then swaps them (wavefront.cu)
template <typename T>
rbgs_status launch_wavefront_pass(ColourField<T> &fld, int k, cudaStream_t s);
// nsweeps FP64 sweeps of fld in cooperative launches with a bounded grid barrier between
// the colours (persistent.cu); a barrier that gives up sets *status
template <typename T>
rbgs_status launch_persistent_sweeps(ColourField<T> &fld, long nsweeps, unsigned *counter, int *status,
                                     cudaStream_t s);
// FP32 inner sweeps in one launch of one thread-block cluster, d held in its shared memory
// (cluster_sweeps.cu); usable when d of an n^2 grid with row pitch W fits the cluster
bool cluster_sweeps_f32_fit(int n, int W);
rbgs_status launch_cluster_sweeps_f32(ColourField<float> &fld, long nsweeps, cudaStream_t s);
// mixed-precision refinement kernels (mixed.cu)
rbgs_status launch_defect(const rbgs_ctx *c, bool write_r32, double scale, cudaStream_t s);  // -> dsum[0] sum, dsum[2] max
rbgs_status launch_correct(const rbgs_ctx *c, double scale, cudaStream_t s);
// fused FP64 update (fused.cu): max |h2 f| of a loaded problem; the scale of a block of
// nsweeps sweeps with h2 f on its grid; one half-sweep at that scale
rbgs_status launch_fused_rhs_max(const rbgs_ctx *c, cudaStream_t s);
rbgs_status launch_fused_prepare(const rbgs_ctx *c, long long nsweeps, cudaStream_t s);
rbgs_status launch_fused_half_sweep(const rbgs_ctx *c, int colour, cudaStream_t s);

}  // namespace rbgs
