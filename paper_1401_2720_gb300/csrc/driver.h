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
    // false when every Buffer points into memory the context does not own
    // (the no-allocation entry point): nothing is then freed on destruction
    bool owns_memory = true;
    std::string last_error;

    // workspace (grown on demand, freed with the context)
    Buffer g, v, part, vprime, vflag, counters, sigma, border, perm;
    Buffer bslice, bexp, dexp, gexp;
    Buffer dyn_tab, dyn_norm;              // dynamic block ordering: sweep table + permutation, block norms       // split right factors, column exponent bounds (tensor-core contractions)
    Buffer g32, v32, tmp_a, tmp_b, tmp_g;  // mixed precision
    Buffer b_mats, b_units, b_g, b_v, b_part, b_vp, b_vflag, b_tab, b_cnt, b_stat, b_starts, b_sigma,
        b_border, b_perm, b_misc, b_bsl, b_bex, b_dex, b_gexp;   // batched solver
    Buffer adj_w, adj_meta, adj_desc;      // adjoint
    Buffer q_meta, q_w, q_tau, q_piv, q_in, q_u, q_s, q_v;   // batched QR preprocessing
    std::vector<unsigned char> q_meta_host;
    unsigned long long *host_counters = nullptr;  // pinned
    std::map<std::pair<int, int>, Buffer> tables;  // (strategy, order) -> device table
    std::map<std::pair<int, int>, std::vector<int>> host_tables;
    std::map<int, std::vector<unsigned char>> host_inner;  // inner tables (source of their async upload)

    // instrumentation (jsvd_profile)
    bool profiling = false;
    static constexpr int kClasses = 5;   // Gram, Jacobi, update (main stream), V update (side stream), other
    double prof_ms[kClasses] = {0, 0, 0, 0, 0};
    long long prof_launches[kClasses] = {0, 0, 0, 0, 0};
    double prof_flops[kClasses] = {0, 0, 0, 0, 0};
    std::vector<cudaEvent_t> events;  // 6 per p-step of one sweep
    int ensure_events(size_t count);

    // The V update of a p-step runs on a side stream; V' lives in a ring of
    // kVRing slots guarded by events (no device-side waits).
    static constexpr int kVRing = 4;
    bool side_streams = true;
    cudaStream_t vstream = nullptr;        // least priority: V updates
    cudaStream_t mstream = nullptr;        // greatest priority: everything else of a solve
    std::vector<cudaEvent_t> ring_events;  // [0, ring): Jacobi done, [ring, 2 ring): V update done,
                                           // [2 ring]: join, [2 ring + 1]: fork/join with the caller
    int ensure_side_stream();

    virtual ~jsvd_ctx();
    void release_memory();   // cudaFree / cudaFreeHost of every Buffer, table and the pinned counters
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
    int solve_batched_qr(int batch, const int *m, const int *n, const int *b, const double *A,
                         const long long *a_off, double *S, const long long *s_off, double *U,
                         const long long *u_off, double *V, const long long *v_off, const jsvd_opts *opts,
                         jsvd_info *infos);
    int backward(int batch, const int *m, const int *n, const double *U, const long long *u_off,
                 const double *S, const long long *s_off, const double *V, const long long *v_off,
                 const double *dU, const double *dS, const double *dV, double *dA, const long long *a_off);
    int solve_on_stream(int m, int n, int nplus, const double *A, int lda, double *S, double *U, int ldu,
                        double *V, int ldv, const jsvd_opts *opts, jsvd_info *info, bool hyperbolic);
    int solve(int m, int n, int nplus, const double *A, int lda, double *S, double *U, int ldu,
              double *V, int ldv, const jsvd_opts *opts, jsvd_info *info, bool hyperbolic);
    int block_pstep(int m, int n, int b, int strategy, int step, double *G, int ldg, double *V, int ldv,
                    int contraction, jsvd_info *info);
};
