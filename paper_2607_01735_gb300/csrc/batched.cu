// Batched solve of independent problems.
#include <cmath>
#include "common.cuh"

extern "C" rbgs_status rbgs_solve_batched(int nprob, const rbgs_problem *probs, double tol,
                                          const rbgs_opts *opts, void *cuda_stream,
                                          double **u_out, rbgs_result *res) {
    rbgs::clear_error();
    if (nprob < 0 || (nprob > 0 && (!probs || !u_out || !res))) {
        rbgs::set_error("bad batched arguments");
        return RBGS_EINVAL;
    }
    rbgs_status first = RBGS_OK;
    for (int p = 0; p < nprob; ++p) {
        rbgs_t c = nullptr;
        rbgs_status st = rbgs_create(probs[p].n, probs[p].h2, probs[p].f, probs[p].u_init, opts,
                                     cuda_stream, &c);
        long sweeps = 0;
        double rel = NAN;
        if (st == RBGS_OK) st = rbgs_solve(c, tol, &sweeps, &rel);
        if (st == RBGS_OK || st == RBGS_ENOTCONV) {
            rbgs_status g = rbgs_get_solution(c, u_out[p]);
            if (g != RBGS_OK) st = g;
        }
        rbgs_destroy(c);
        res[p].status = st;
        res[p].sweeps = sweeps;
        res[p].rel = rel;
        res[p].latency_ms = 0.0;
        if (st != RBGS_OK && first == RBGS_OK) first = st;
    }
    return first;
}
