// Host-side context of the C ABI: device copies of the gauge field and clover
// terms per storage precision, the gauge-state generation counter (Sec. 3's
// gauge_id cascade), reduction scratch and solver workspace.
#pragma once

#include <map>
#include <string>

#include "tm_internal.h"
#include "tm_kernels.h"

struct tm_ctx {
    // unique over the process lifetime (a destroyed context's address can be reused
    // by the next one, so caches keyed on derived state use this id, not the pointer)
    unsigned long long uid = 0;
    int device = 0;
    tmk::Geom g{};
    long vh = 0;
    cudaStream_t sstream = nullptr;   // private stream for solver work (graph capture)

    // gauge state (Sec. 3: tm_GaugeState_t / update_tm_gauge_id)
    double gauge_id = 0.0;
    long gauge_gen = 0;                // 0 = no gauge loaded
    void* gauge64[2] = {nullptr, nullptr};
    void* gaugeP[4][2] = {};
    long gaugeP_gen[4] = {0, 0, 0, 0};

    // clover state: computed for (gauge_gen, params)
    tm_params params{};
    long clover_gauge_gen = -1;
    long clover_stamp = 0;
    bool have_heavy = false;
    double* clovA64[2] = {nullptr, nullptr};
    double* clovB64 = nullptr;
    double* clovH64 = nullptr;
    void* clovAP[4] = {};
    void* clovBP[4] = {};
    void* clovHP[4] = {};
    long clovP_stamp[4] = {0, 0, 0, 0};
    // double-word copies of the FP64 links and clover arrays (odd A, even light,
    // even heavy) for the reliable updates of the mixed-precision solvers
    void* gaugeDF[2] = {nullptr, nullptr};
    long gaugeDF_gen = 0;
    void* clovDF[3] = {};
    long clovDF_stamp = 0;
    // even-site A in a storage precision, made only for the full operator (multigrid)
    void* clovAeP[4] = {};
    long clovAeP_stamp[4] = {0, 0, 0, 0};

    // reduction scratch and control words
    double* partial = nullptr;
    unsigned int* counter = nullptr;
    int max_blocks = 0;
    tmk::SolverCtl* ctl = nullptr;
    tmk::MsCtl* ms = nullptr;
    tmk::SolverCtl* h_ctl = nullptr;   // pinned mirrors
    tmk::MsCtl* h_ms = nullptr;
    double* d_scal = nullptr;          // 16 FP64 reduction results
    double* h_scal = nullptr;

    std::map<int, std::pair<void*, size_t>> ws;   // workspace buffers by id

    // host-buffer staging of tm_field_import / tm_field_export: a ring of device
    // buffers per direction, each released by an event recorded after its last use,
    // so calls with pinned host memory on different streams can overlap
    struct IoRing {
        static constexpr int N = 3;
        void* buf[N] = {};
        cudaEvent_t free[N] = {};
        size_t bytes = 0;
        int next = 0;
    } io_in, io_out;

    // stencil kernel variant per [storage precision][flavours - 1][pass]:
    // 0 = direct (registers), 1 = shared-memory staged; set by tm_autotune / tm_set_tuning
    int variant[4][2][2] = {};
};
