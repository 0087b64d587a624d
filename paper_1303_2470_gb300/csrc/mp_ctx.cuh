// mp_ctx.cuh -- the MP context behind the opaque mp_ctx handle of the C ABI, shared by the
// translation units of libmp (not part of the C ABI), and the entry points of the direct
// scheme (mp_direct.cu) that the context and group functions call.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "internal.cuh"

struct mp_group;

namespace mp {
struct DirectTables;
struct DirectState;
}  // namespace mp

struct mp_ctx {
    mp::Geometry geo;
    int precision = MP_FP32;
    int S = 0, F = 0, M = 0;
    int dir[3] = {0, 0, 0};
    cudaStream_t stream = nullptr;
    long long cap = 0;
    long long t = 0;
    double Db[MP_MAX_SPECIES], ka[MP_MAX_SPECIES], kd[MP_MAX_SPECIES];
    void* u4 = nullptr;          // Flow4<T> per node
    uint32_t* fmask = nullptr;   // open-link mask per fluid node
    void* P[2] = {nullptr, nullptr};
    void* A[2] = {nullptr, nullptr};
    int cur = 0;
    double* Z = nullptr;
    double* D = nullptr;
    long long* tdev = nullptr;
    double* partials = nullptr;
    unsigned int* ticket = nullptr;
    int blocks = 0;
    long long n_neg_links = 0, n_neg_stay = 0;
    std::vector<int32_t> ilist;
    size_t elem = 4;
    int FP = 2;  // fields per species record (F padded to 2 or 4)
    int SP = 1;  // species padded to whole chunks (1 for one species)
    int SC = 1;  // species per chunk
    // free fields stored over the fluid list only ([chunk][k][record], k the index in the
    // sorted fluid list) instead of over every lattice node: direct scheme, several species
    bool compact = false;
    std::vector<int32_t> hflist;  // host copy of the fluid list (field I/O of compact fields)
    mp_group* owner = nullptr;  // set while the context steps as part of a group
    double zsc[MP_MAX_SPECIES] = {};  // stored value x zsc = field value (binary16 storage)
    int stochastic = 1;               // binary16 rounding: stochastic (1) or to nearest (0)
    // runs of kCtxGraphSteps steps captured once per starting buffer (cur) and replayed
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    // direct scheme (MP_SCHEME_DIRECT): per-node tables, and the launch state that steps this
    // context on its own (both built by mp_init)
    int scheme = MP_SCHEME_FLUX;
    mp::DirectTables* dtab = nullptr;
    mp::DirectState* dstate = nullptr;
};

namespace mp {

// Direct scheme (mp_direct.cu). direct_setup builds c->dtab and c->dstate after the fields are
// initialised (tune != 0: time the kernel variants on the current state and keep the fastest;
// otherwise run `variant`, MP_VARIANT_* flags);
// direct_step advances the context n steps on its own stream; direct_check reports a bounded
// device wait that gave up (MP_ETIMEOUT) and clears it (synchronises the stream).
int direct_setup(mp_ctx* c, int tune, int variant);
int direct_step(mp_ctx* c, long long n);
int direct_check(mp_ctx* c);
void direct_free(mp_ctx* c);

// A set of direct-scheme contexts stepped together (groups): created over n contexts, run on
// `stream`, stepped n steps; variant and block size are autotuned when `tune` is nonzero.
int direct_state_create(mp_ctx* const* ctxs, int n, cudaStream_t stream, int tune, int variant,
                        DirectState** out);
int direct_state_step(DirectState* d, long long n);
int direct_state_check(DirectState* d);
void direct_state_free(DirectState* d);
const char* direct_state_variant(const DirectState* d);
int direct_state_block(const DirectState* d);

}  // namespace mp
