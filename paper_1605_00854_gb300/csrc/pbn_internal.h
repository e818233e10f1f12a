/* pbn_internal.h -- host-side model and plan objects shared by the library's
 * C++ preparation code and its CUDA launch code. */
#ifndef PBN_INTERNAL_H
#define PBN_INTERNAL_H

#include <cstdint>
#include <string>
#include <vector>

#include "pbn.h"
#include "pbn_image.h"

struct pbn_fun {
    double c = 0.0;                 /* selection probability */
    std::vector<uint32_t> par;      /* parents a_0..a_{k-1} */
    std::vector<uint64_t> tt;       /* 2^k output bits, bit x in word x / 64 */
    bool bit(uint64_t x) const { return (tt[x >> 6] >> (x & 63)) & 1u; }
};

struct pbn_net {
    uint32_t n = 0;
    double p = 0.0;
    std::vector<std::vector<pbn_fun>> node;   /* node[i][j] = f_{j+1}^{(i)} */
    std::vector<uint8_t> retained;             /* 1 = simulated */
    std::vector<uint32_t> interest;            /* nodes of interest given to pbn_reduce */
};

struct pbn_jit_state;

struct pbn_plan {
    pbn_plan_info info{};
    pbn_img_header hdr{};
    std::vector<uint8_t> image;      /* device image, 16-byte padded */
    std::vector<uint32_t> pos;       /* per original node: 32 * row + bit, or UINT32_MAX */
    std::vector<uint32_t> group_of;  /* per original node: group index, or UINT32_MAX */
    uint32_t per_traj_smem = 0;      /* shared-memory bytes per trajectory slot */
    mutable pbn_jit_state* jit = nullptr; /* compiled-plan cache (pbn_jit.cpp) */
    ~pbn_plan();
};

struct pbn_jit_params_s;

namespace pbn {
int fail(int code, const char* fmt, ...);
uint64_t pert_threshold(double p);

/* The meta-state as state rows: for each 32-bit row of the plan's state that holds
 * one of the n_meta nodes, the row index, the mask of those nodes and the values they
 * must take (vals NULL: all 1).  At most max_rows rows.  Errors (PBN_EINVAL, the
 * message prefixed by `who`): a node that is not retained, more than max_rows rows,
 * one node listed with two different values. */
struct MetaRows {
    uint32_t n_rows = 0;
    uint32_t row[64], mask[64], val[64];
};
int meta_rows(const pbn_plan* plan, const uint32_t* ids, const uint8_t* vals, uint32_t n_meta, uint32_t max_rows,
              const char* who, MetaRows* out);
/* compiled plans (pbn_jit.cpp) */
pbn_jit_state* jit_state(const pbn_plan* plan);
void jit_free(pbn_jit_state* J);
int jit_compile(const pbn_plan* plan, uint32_t flags);
bool jit_ready(const pbn_plan* plan);
uint32_t jit_current_flags(const pbn_plan* plan); /* flags of the compiled kernel, else 0 */

/* Compiled networks of a batch (pbn_jit.cpp): what a network fixes at generation
 * time, its device function, and the batch module of such functions and the
 * persistent dispatcher kernel. */
struct JitBatchNet {
    uint32_t index = 0;  /* position in the batch: the function is pbn_net_<index> */
    uint64_t seed = 0;   /* Philox key of the network's draws */
    MetaRows meta;       /* the network's meta-state rows */
};
/* Source of network `spec.index`'s work-item function and the bytes of its tables to
 * stage into shared memory (0: read from the plan image); false, with the reason,
 * if the plan does not compile with these flags. */
bool jit_batch_function(const pbn_plan* plan, uint32_t flags, const JitBatchNet& spec, std::string* src,
                        uint32_t* tab_bytes, std::string* why);
/* Compile the module of `functions` (one per network in `compiled`, in parallel
 * relocatable units) and a persistent kernel of `threads` threads per CTA dispatching
 * work items to pbn_net_<i> and, when `interp`, to the interpreter's relocatable
 * work-item function; link them with nvJitLink and load the result.
 * Errors: PBN_ECUDA (NVRTC, nvJitLink or loading failed; *log holds the reason). */
int jit_batch_module(const std::vector<std::string>& functions, const std::vector<uint32_t>& compiled, bool interp,
                     uint32_t threads, void** library, void** kernel, double* ms, std::string* log);
void jit_library_unload(void* library);

/* Launch facts of the current device, queried once per device (thread-safe). */
int device_sms();         /* SM count */
int device_smem_optin();  /* opt-in dynamic shared memory per block, bytes */
/* Raise `func`'s dynamic shared-memory limit on the current device to at least
 * `bytes` when `bytes` plus the kernel's static shared memory (`static_bytes`, an
 * upper bound is enough; the library's kernels hold less than the default) exceeds
 * the 48 KB a launch gets without opting in; the limit is per device and per kernel
 * and is only ever raised, so that callers sharing a kernel never lower each other's
 * setting.  Returns a cudaError_t value (0 = success). */
int ensure_dyn_smem(const void* func, size_t bytes, size_t static_bytes = 1024);
}  // namespace pbn

#endif
