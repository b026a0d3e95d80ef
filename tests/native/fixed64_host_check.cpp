// Host harness for the fused update's fixed-point helpers (csrc/fixed64.cuh): exposes them
// over a C interface so the CPU test suite can compare them with exact conversions.  Test
// infrastructure only.
#include <cmath>

#include "../../paper_2607_01735_gb300/csrc/fixed64.cuh"

extern "C" {

void check_to_fixed(long n, const double *t, const int *e, long long *out) {
    for (long q = 0; q < n; ++q) out[q] = (long long)rbgs::to_fixed(t[q], e[q]);
}

void check_fixed_quarter(long n, const long long *s, const int *e, double *out) {
    for (long q = 0; q < n; ++q) out[q] = rbgs::fixed_quarter_to_double((int64_t)s[q], e[q]);
}

// e, or -100000 when scale_exponent reports a non-finite bound
void check_scale_exponent(long n, const double *B, const double *Q, const long long *sweeps, int *out) {
    for (long q = 0; q < n; ++q) {
        int e = 0;
        out[q] = rbgs::scale_exponent(B[q], Q[q], sweeps[q], &e) ? e : -100000;
    }
}

}
