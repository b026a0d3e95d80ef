// Layout conversion between the caller's natural grid and the colour-split layout
// (red/black split storage, Section 2.1 of the paper).  Each thread handles the natural
// pair of columns (2k, 2k+1) of one row: one of them is red and the other black, and in
// the colour-split layout both sit at element k of their colour's row.
#include "common.cuh"

namespace rbgs {
namespace {

constexpr int kThreads = 256;

// u_nat: (n+2) x (n+2) natural grid -> colour rows of width W (padding set to zero).
__global__ void pack_u_kernel(const double *__restrict__ u_nat, double *__restrict__ red,
                              double *__restrict__ black, int n, int W) {
    const int k = blockIdx.x * kThreads + threadIdx.x;
    if (k >= W) return;
    const int ld = n + 2;
    for (int i = blockIdx.y; i < n + 2; i += gridDim.y) {
        const int j = 2 * k;
        const double a = (j <= n + 1) ? u_nat[(size_t)i * ld + j] : 0.0;
        const double b = (j + 1 <= n + 1) ? u_nat[(size_t)i * ld + j + 1] : 0.0;
        double *even_dst = (i & 1) ? black : red;   // colour of (i, 2k) is i & 1
        double *odd_dst = (i & 1) ? red : black;
        even_dst[(size_t)i * W + k] = a;
        odd_dst[(size_t)i * W + k] = b;
    }
}

// f_nat: n x n interior -> h2*f in colour rows (zero on the ring and in the padding).
// h2*f is one correctly rounded product, the value the update's first term needs.
__global__ void pack_f_kernel(const double *__restrict__ f_nat, double h2,
                              double *__restrict__ hf_red, double *__restrict__ hf_black, int n,
                              int W) {
    const int k = blockIdx.x * kThreads + threadIdx.x;
    if (k >= W) return;
    for (int i = blockIdx.y; i < n + 2; i += gridDim.y) {
        const bool row_in = (i >= 1 && i <= n);
        const int j = 2 * k;
        const double a = (row_in && j >= 1 && j <= n)
                             ? __dmul_rn(h2, f_nat[(size_t)(i - 1) * n + (j - 1)]) : 0.0;
        const double b = (row_in && j + 1 <= n)
                             ? __dmul_rn(h2, f_nat[(size_t)(i - 1) * n + j]) : 0.0;
        double *even_dst = (i & 1) ? hf_black : hf_red;
        double *odd_dst = (i & 1) ? hf_red : hf_black;
        even_dst[(size_t)i * W + k] = a;
        odd_dst[(size_t)i * W + k] = b;
    }
}

__global__ void unpack_u_kernel(const double *__restrict__ red, const double *__restrict__ black,
                                double *__restrict__ u_nat, int n, int W) {
    const int k = blockIdx.x * kThreads + threadIdx.x;
    const int j = 2 * k;
    if (j > n + 1) return;
    const int ld = n + 2;
    for (int i = blockIdx.y; i < n + 2; i += gridDim.y) {
        const double *even_src = (i & 1) ? black : red;
        const double *odd_src = (i & 1) ? red : black;
        u_nat[(size_t)i * ld + j] = even_src[(size_t)i * W + k];
        if (j + 1 <= n + 1) u_nat[(size_t)i * ld + j + 1] = odd_src[(size_t)i * W + k];
    }
}

dim3 layout_grid(const Geometry &g) {
    int gy = g.rows < 65535 ? g.rows : 65535;
    return dim3((g.W + kThreads - 1) / kThreads, gy);
}

}  // namespace

rbgs_status launch_pack_u(const Geometry &g, const double *u_nat, double *red, double *black,
                          cudaStream_t s) {
    pack_u_kernel<<<layout_grid(g), kThreads, 0, s>>>(u_nat, red, black, g.n, g.W);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

rbgs_status launch_pack_f(const Geometry &g, double h2, const double *f_nat, double *hf_red,
                          double *hf_black, cudaStream_t s) {
    pack_f_kernel<<<layout_grid(g), kThreads, 0, s>>>(f_nat, h2, hf_red, hf_black, g.n, g.W);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

rbgs_status launch_unpack_u(const Geometry &g, const double *red, const double *black,
                            double *u_nat, cudaStream_t s) {
    unpack_u_kernel<<<layout_grid(g), kThreads, 0, s>>>(red, black, u_nat, g.n, g.W);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

}  // namespace rbgs
