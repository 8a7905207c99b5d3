// The context object behind jsvd_ctx_t.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <utility>
#include <vector>

#include "jsvd.h"

struct Buffer {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct jsvd_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool verbose = false;
    std::string last_error;

    // workspace (grown on demand, freed with the context)
    Buffer g, v, part, vprime, vflag, counters, sigma, border, perm;
    Buffer g32, v32, tmp_a, tmp_b, tmp_g;  // mixed precision
    Buffer b_mats, b_units, b_g, b_v, b_part, b_vp, b_vflag, b_tab, b_cnt, b_stat, b_starts, b_sigma,
        b_border, b_perm, b_misc;          // batched solver
    Buffer adj_w, adj_meta, adj_desc;      // adjoint
    unsigned long long *host_counters = nullptr;  // pinned
    std::map<std::pair<int, int>, Buffer> tables;  // (strategy, order) -> device table
    std::map<std::pair<int, int>, std::vector<int>> host_tables;

    // instrumentation (jsvd_profile)
    bool profiling = false;
    double prof_ms[4] = {0, 0, 0, 0};
    long long prof_launches[4] = {0, 0, 0, 0};
    double prof_flops[4] = {0, 0, 0, 0};
    std::vector<cudaEvent_t> events;  // 4 per p-step of one sweep
    int ensure_events(size_t count);

    virtual ~jsvd_ctx();
    void set_error(const char *where, cudaError_t e);
    int check(const char *where);
    int sync(const char *where);
    int polar_and_apply(double *G, int ldg, int n, int nplus, const float *V32, int ldv32, double *V, int ldv);
    virtual int ensure(Buffer &buf, size_t bytes);
    int table(int strategy, int n, const int **dev);
    int inner_table(int strategy, int BB, const unsigned char **dev);
    int solve_batched(int batch, const int *m, const int *n, const int *b, const double *A,
                      const long long *a_off, double *S, const long long *s_off, double *U,
                      const long long *u_off, double *V, const long long *v_off, const jsvd_opts *opts,
                      jsvd_info *infos);
    int backward(int batch, const int *m, const int *n, const double *U, const long long *u_off,
                 const double *S, const long long *s_off, const double *V, const long long *v_off,
                 const double *dU, const double *dS, const double *dV, double *dA, const long long *a_off);
    int solve(int m, int n, int nplus, const double *A, int lda, double *S, double *U, int ldu,
              double *V, int ldv, const jsvd_opts *opts, jsvd_info *info, bool hyperbolic);
};
