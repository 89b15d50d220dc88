// Host-side plan object and the internal host functions shared by the
// plan, batch and serving code.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/slp.h"
#include "../../include/slp_debug.h"
#include "slp_internal.h"

// Auxiliary stream and fork/join events of one execution context: the
// near-field branch runs on `aux` while the far-field chain runs on the
// caller's stream.
struct SlpExec {
    cudaStream_t aux = nullptr;
    // the spread / FFT / gather chain runs on `main` (highest priority), so
    // its blocks are dispatched ahead of the near-field branch's when both
    // are pending; `done` returns the chain to the caller's stream
    cudaStream_t main = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, done = nullptr;
    // optional timeline (5 events): start, spread done, FFT passes done (on
    // the caller's stream), near branch done (auxiliary stream), gather done
    cudaEvent_t *timeline = nullptr;
};
cudaError_t slp_exec_create(SlpExec &e);
void slp_exec_destroy(SlpExec &e);

struct slp_plan_s {
    // configuration
    slp_plan_opts opts;
    int q = 0;
    int prec = 32;
    double tol = 0;
    int64_t N = 0, M = 0, Q = 0;
    int device = 0;

    // geometry (host, FP64)
    std::vector<double> V;       // [N][3]
    std::vector<int32_t> T;      // [M][3]
    std::vector<double> lam, wq; // rule
    std::vector<double> y;       // [Q][3] user order
    std::vector<double> wk;      // [Q]
    std::vector<double> nrm;     // [M][3]

    // parameters
    int L[3] = {0, 0, 0}, n[3] = {0, 0, 0}, m = 0, TS = 8, TE = 0;
    int TSg = 8;  // target (gather) tile size in cells
    int gather_chunk = 64;  // most targets in one gather item
    int kf = 1;   // states of one far-field batch (scratch copies per scratch set)
    int kernel_mode = SLP_KERNEL_RADIAL, near_mode = SLP_NEAR_ON_THE_FLY;
    int grid_raised = 0;
    double ctr[3] = {0, 0, 0}, P[3] = {0, 0, 0}, D[3] = {0, 0, 0};
    double diam = 0, sigma_g = 0, R = 0, eps = 0, c_band = 0;
    double sep_A = 0;
    std::vector<double> sep_h[3];
    // EXPSUM: kept terms w_k exp(-g_k u^2) of 1/u in torus units (u = r / P),
    // and per axis the one-period Fourier factors I_k(l), [S'][n_q / 2]
    std::vector<double> es_w, es_g, es_I[3];
    // triangle-integrated plans: entries of the gridding and near-field matrices
    int64_t am_nnz = 0, nt_nnz = 0;

    // sorted data (host)
    std::vector<int32_t> src_perm, tgt_perm;
    std::vector<double> src_grid, tgt_grid;  // [.][4]
    std::vector<slp::TileItem> spread_items, gather_items;
    std::vector<int32_t> sgroups, sgroup_off;  // spread cell groups and per-item warp lists
    std::vector<int32_t> sgroup_cell;          // local cell of each group (lx | ly << 8 | lz << 16)
    std::vector<slp::NearItem> near_items;
    std::vector<int2> near_ranges;
    std::vector<int> near_blk_first;  // CSR of items per target block
    std::vector<double> Dtab;
    int64_t near_pairs = 0;
    // rows of the grid the FFT passes work on: the cyclic z interval
    // [z0, z0 + nz_act) and, per plane, a pair-aligned cyclic y interval
    std::vector<int2> plane_iv;       // [Lz] (y0, rows)
    std::vector<int32_t> row_pairs;   // z * (Ly / 2) + y / 2 of each active row pair
    int z0 = 0, nz_act = 0;

    // device
    slp::DevPlan dp;
    std::vector<void *> allocs;
    int64_t bytes_device = 0;
    void *d_stage_in = nullptr, *d_stage_phi = nullptr;
    // pipelined host-buffer evaluations: two staging slots, copy streams and
    // the events that order them (copy-in k -> evaluation k -> copy-out k)
    void *d_astage_in[2] = {nullptr, nullptr}, *d_astage_phi[2] = {nullptr, nullptr};
    cudaStream_t cs_in = nullptr, cs_out = nullptr;
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_eval[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
    int aslot = 0;
    int *d_blk_first = nullptr;
    int launches_per_eval = 0;
    int64_t near_pairs_within = -1;
    int64_t nm_nnz = 0;
    SlpExec exec;  // for evaluations on the plan's own scratch
};


// Record a failure text for slp_last_error() and return the status.
slp_status slp_fail(slp_status st, const char *fmt, ...);

// Values of one input of the given kind (SLP_INPUT_*).
inline int64_t slp_input_count(const slp_plan_s &p, int kind) {
    switch (kind) {
        case SLP_INPUT_SIGMA: return p.Q;
        case SLP_INPUT_MAG: return 3 * p.Q;
        case SLP_INPUT_NODAL_MAG: return 3 * p.N;
        case SLP_INPUT_ELEMENT: return p.M;
    }
    return 0;
}

// SLP_OK when the plan evaluates inputs of this kind.
slp_status slp_check_kind(const slp_plan_s &p, int kind);

// Events of a profiled evaluation: kernel slot i is bracketed by ev[2i] and
// ev[2i + 1] on its launch stream, and launched[i] is set when it ran.
constexpr int SLP_PROFILE_SLOTS = 15;
struct SlpProfile {
    cudaEvent_t ev[2 * SLP_PROFILE_SLOTS];
    bool launched[SLP_PROFILE_SLOTS];
};

// Enqueue one evaluation of `p` with the device view `d` (the plan's own
// scratch or another scratch set) up to stage `last`.  With ex != NULL (and
// no profile) the near-field branch runs concurrently on ex->aux; with prof
// != NULL everything runs in order on s and each launched kernel is timed.
slp_status slp_run_pipeline(slp_plan_s &p, const slp::DevPlan &d, int kind, const void *d_in, void *d_phi,
                            cudaStream_t s, int last, SlpProfile *prof, SlpExec *ex);

// Enqueue n evaluations of `p` on the device view `d` (states ins[k] ->
// outs[k]); nodal input with the precomputed near field shares one pass over
// the near-field operator among up to NEAR_STATES states.  Adds the kernels
// launched to *launches when given.
slp_status slp_run_states(slp_plan_s &p, const slp::DevPlan &d, int kind, const void *const *ins, void *const *outs,
                          int n, cudaStream_t s, SlpExec *ex, int *launches);

// Allocate a second scratch set (charges, sorted m, grids, spectra, partials)
// for `p` and return a device view that uses it; the pointers are appended to
// `allocs` (released by the caller with cudaFree).  Grids and spectra are
// zeroed (rows outside the active region are never written afterwards).
slp_status slp_alloc_scratch(slp_plan_s &p, slp::DevPlan &out, std::vector<void *> &allocs, int64_t *bytes);

// Release the graphs slp_eval_batched cached for argument sets that use `plan`
// (called by slp_destroy).
void slp_batch_cache_drop(const slp_plan_s *plan);

// Bytes of one scratch set of `p`.
int64_t slp_scratch_bytes(const slp_plan_s &p);

// States of one far-field batch: the spread, FFT and gather scratch is held
// this many times (at most NEAR_STATES, within 2 GB per scratch set).
int slp_far_batch(const slp_plan_s &p);

// Current device switched to `dev` for the guard's lifetime.
struct SlpDeviceGuard {
    int prev = -1;
    explicit SlpDeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (dev >= 0 && prev != dev) cudaSetDevice(dev);
    }
    ~SlpDeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};
