// handle.hpp -- the gmres_handle structure shared by the library's
// translation units (solver driver, learned preconditioner): device copies of
// A, the workspace, the control block and the per-class event timer.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <vector>

#include "common.cuh"
#include "host_util.hpp"

namespace gmres_host {

// Event pairs for per-class kernel timing (opts.profile).
struct Timer {
    bool on = false;
    cudaStream_t st = nullptr;
    std::vector<cudaEvent_t> pool;
    struct Rec { int cls; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    cudaEvent_t begin() {
        if (!on)
            return nullptr;
        cudaEvent_t a = get();
        cudaEventRecord(a, st);
        return a;
    }
    void end(int cls, cudaEvent_t a) {
        if (!on)
            return;
        cudaEvent_t b = get();
        cudaEventRecord(b, st);
        recs.push_back({cls, a, b});
    }
    // after a stream synchronize
    void harvest(double *ms) {
        for (auto &r : recs) {
            float t = 0;
            if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess)
                ms[r.cls] += t;
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        recs.clear();
    }
    void destroy() {
        for (auto &r : recs) {
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        recs.clear();
        for (auto e : pool)
            cudaEventDestroy(e);
        pool.clear();
    }
};

}  // namespace gmres_host

struct gmres_handle {
    using DevBuf = gmres_host::DevBuf;
    using Timer = gmres_host::Timer;
    int n = 0;
    int64_t nnz = 0;
    int64_t ldv = 0;
    int device = 0;
    int nsm = 0;
    cudaStream_t stream = nullptr;
    gmres_opts opts;
    int lanes32 = 4, lanes64 = 4;
    int grid = 0;          // blocks of the reduction kernels
    int rows_blocks_per_sm = 4;  // blocks per SM of the register-streaming CGSR kernels
    int64_t mgs_chunk = 0;       // rows per block of the cooperative MGS kernel
    int64_t mgss_chunk = 0;      // rows per block of the staged cooperative MGS kernel
    std::map<const void *, bool> mgs_ok_cache;  // cooperative MGS feasible, per kernel
    DevBuf mgs_seq;              // exchange slots of the cooperative MGS kernel
    DevBuf mon;                  // restart-test histories and the U, S matrices
    bool limited = false;        // the running solve is GMRES_MIXED_LIMITED
    bool split = false;          // A stored split: vals64 holds hi[nnz] then lo[nnz]
    int work_elem = 0;           // bytes of the working type the work vectors last held
    // ILU(0) left preconditioner: factors (binary64 and binary32 copies),
    // diagonal positions, ready flags of the two triangles + claim counters
    DevBuf ilu64, ilu32, ilu_dpos, ilu_flags, t2;
    DevBuf ilu_order;            // rows in level order: L's n entries, then U's
    DevBuf ilu_lptr;             // level starts in ilu_order: L's levels + 1, then U's
    int ilu_ok = 0;
    int ilu_levels = 0;
    int ilu_ulevels = 0;
    bool ilu_wave_ok[2] = {false, false};  // L, U suit the barrier-free solve
    unsigned ilu_epoch = 1;
    unsigned mgs_round = 0;      // next exchange round number (0: flags not set up)
    int64_t chunk = 0;     // rows per block
    // matrix
    DevBuf rowptr, colind, vals64, vals32;
    // A in sliced storage (sell.cuh): slice offsets, row lengths, columns
    // (16-bit offsets from the row or 32-bit), binary32 and binary64 values;
    // built by gmres_autotune or on request (gmres_opts.spmv_format)
    DevBuf sptr, slen, scol, sval32, sval64;
    int sell_fmt = 0;             // 0: not built, 1: 16-bit offsets, 2: 32-bit columns
    int64_t sell_entries = 0;     // entries stored, padding included
    bool sell32 = false, sell64 = false;  // the autotuner chose it (binary32 / binary64)
    DevBuf trowptr, tcolind, tvals64;  // A^T (optional)
    // workspace
    DevBuf V, w, r, t, z, xb, bb;
    DevBuf small;          // H, Hb, s, cs, sn, y, h1, h2
    DevBuf part, part64, ctl;
    DevBuf bsys, bres;     // block-solver descriptor / result
    gmres::Ctl *hctl = nullptr;   // pinned copy of the control block
    Timer timer;
    // learned right preconditioner on A's pattern (binary64 / binary32 values)
    DevBuf pvals64, pvals32;
    int has_precond = 0;
    // learned-preconditioner workspace: features (9 x nnz), per-row stats,
    // binary32 A^T values, parameters, M, dL/dm, activations, vectors,
    // partial sums, probes, gradient
    DevBuf spai_feat, spai_rowv, tvals32, spai_params, spai_m, spai_gm, spai_H, spai_vec,
        spai_part, spai_Z, spai_grad;
    int spai_feat_ok = 0;
};
