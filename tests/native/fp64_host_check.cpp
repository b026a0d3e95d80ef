// Host harness for the library's exact binary64 helpers (csrc/fp64.cuh): exposes them
// over a C interface so the CPU test suite can compare them with the CPU's own IEEE
// addition and multiplication.  Test infrastructure only.
#include "../../paper_2607_01735_gb300/csrc/fp64.cuh"
#include "../../paper_2607_01735_gb300/csrc/div6.cuh"

extern "C" {

void check_add_int(long n, const double *a, const double *b, double *out) {
    for (long q = 0; q < n; ++q) out[q] = rbgs::add_int(a[q], b[q]);
}

// the integer path alone: ok[q] = 1 where it applies (its result must then be exact)
void check_add_core(long n, const double *a, const double *b, double *out, int *ok) {
    for (long q = 0; q < n; ++q) {
        bool k;
        out[q] = rbgs::add_int_core(a[q], b[q], k);
        ok[q] = k ? 1 : 0;
    }
}

void check_div6(long n, const double *a, double *out) {
    for (long q = 0; q < n; ++q) out[q] = rbgs::div6(a[q]);
}

void check_quarter(long n, const double *a, double *out) {
    for (long q = 0; q < n; ++q) out[q] = rbgs::quarter(a[q]);
}

}
