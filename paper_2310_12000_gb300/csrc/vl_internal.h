// Internal declarations of libvl: context, workspace arena, handles, launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <map>
#include <tuple>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/vl.h"

namespace vl {

// ----------------------------------------------------------------------------- status
// Device-side status block: the first error code/row wins; `abort` tells every
// bounded wait in a running kernel to give up at once.
struct DevStatus {
  int code;
  int row;
  int abort;
  int pad;
  long long limit;   // cycles a bounded wait may take (0: the default); kept by status_clear
};
constexpr size_t kStatusClearBytes = 4 * sizeof(int);   // code, row, abort, pad

// ----------------------------------------------------------------------------- arena
// First-fit sub-allocator over one device buffer (the caller's workspace).
class Arena {
 public:
  void init(char* base, size_t size);
  void* alloc(size_t bytes);   // nullptr when exhausted
  void release(void* p);
  size_t in_use() const { return in_use_; }
  size_t peak() const { return peak_; }
  size_t size() const { return size_; }

 private:
  char* base_ = nullptr;
  size_t size_ = 0, in_use_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;            // offset -> bytes
  std::unordered_map<size_t, size_t> used_;  // offset -> bytes
};

// Kernel-class timing with CUDA events (enabled by vl_profile_enable).
struct Profiler {
  bool on = false;
  struct Pending {
    std::string key;
    int t;
    cudaEvent_t a, b;
  };
  struct Acc {
    double ms = 0.0;
    int64_t launches = 0;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  std::map<std::pair<std::string, int>, Acc> acc;
  bool trace = false;                                   // record level traces of solves
  long long* dtrace = nullptr;                          // device scratch for one trace
  size_t dtrace_len = 0;
  std::map<std::pair<std::string, int>, std::vector<long long>> traces;   // last per class
  std::map<std::pair<std::string, int>, std::pair<int, int>> cuts;        // (l_head, l_tail)
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool owns_ws = false;
  char* ws = nullptr;
  Arena arena;
  std::string last_error;
  DevStatus* dstatus = nullptr;   // device
  DevStatus* hstatus = nullptr;   // pinned host mirror
  char* pinned = nullptr;         // pinned scratch for small read-backs
  size_t pinned_bytes = 0;
  int num_sms = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t ev_ring[2] = {nullptr, nullptr};   // PCG read-backs one iteration behind
  Profiler prof;
  int64_t launches = 0;           // kernels launched on this context
  unsigned* gbar = nullptr;       // grid-barrier state {count, generation} (device)
  int solve_form = 0;             // vl_solve_form: 0 = chosen per solve, else forced
  bool autotune = true;           // tune result-neutral launch parameters at first use
  int refs = 1;                   // the context itself + every live factor and state
  bool closed = false;            // vl_ctx_destroy was called
};

// Launch-configuration stream argument that also counts the launch.
#define VL_STREAM(c) (++(c)->launches, (c)->stream)

// Brackets the launches issued in its lifetime when profiling is on.
struct ProfScope {
  Ctx* c;
  int idx = -1;
  ProfScope(Ctx* ctx, const char* key, int t);
  ~ProfScope();
};
void prof_drain(Ctx* c);   // resolve finished event pairs (stream must be idle)
void prof_release(Ctx* c); // destroy all events

// RAII list of arena blocks owned by a handle.
struct Owned {
  Ctx* ctx = nullptr;
  std::vector<void*> blocks;
  template <typename T>
  T* get(size_t count) {
    void* p = ctx->arena.alloc(count * sizeof(T) + 16);
    if (p) blocks.push_back(p);
    return static_cast<T*>(p);
  }
  void free_all() {
    for (void* p : blocks) ctx->arena.release(p);
    blocks.clear();
  }
};

struct Factor {
  Ctx* ctx = nullptr;
  Owned mem;
  int64_t n = 0;
  int m = 0;
  // a batch of independent problems merged into one block-diagonal system: problem k owns the
  // storage rows [seg_row0[k], seg_row0[k + 1]); a single problem is one segment
  int nseg = 1;
  std::vector<int64_t> seg_row0;
  int32_t* row_seg = nullptr;   // storage row -> segment (device; batches only)
  int32_t* s2u_loc = nullptr;   // storage row -> caller index within its problem (batches only)
  // caller index that numbers a row's probe and simulation draws (its problem's own index)
  const int32_t* s2u_probe() const { return s2u_loc ? s2u_loc : s2u; }
  int cov = 0;
  double sigma2 = 1.0, rho = 1.0, nugget = 0.0;
  int64_t nnz = 0;            // off-diagonal entries of B
  int nlev_fwd = 0, nlev_bwd = 0;
  // storage order = Morton order of the locations
  double* locs_s = nullptr;   // n x 2
  double* locs_v = nullptr;   // n x 2, Vecchia order
  int32_t* s2v = nullptr;     // storage -> Vecchia index
  int32_t* v2s = nullptr;
  int32_t* s2u = nullptr;     // storage -> caller index
  int32_t* u2s = nullptr;
  int32_t* nbr = nullptr;     // n x m storage indices, -1 padding (ELL of B)
  double* A64 = nullptr;      // n x m kriging weights, B_{i,N(i)} = -A
  float* A32 = nullptr;
  double* D64 = nullptr;      // n
  int32_t* rowptrT = nullptr; // n + 1  (CSR of the transpose pattern)
  int32_t* colT = nullptr;    // nnz: storage row i listing j
  int32_t* permT = nullptr;   // nnz: ELL flat index of the entry
  double* valT64 = nullptr;   // nnz
  float* valT32 = nullptr;
  int32_t* lev_fwd = nullptr; // n (storage order)
  int32_t* lev_bwd = nullptr;
  int32_t* task_fwd = nullptr;  // storage rows sorted by (lev_fwd, s)
  int32_t* task_bwd = nullptr;
  int32_t* lptr_fwd = nullptr;  // nlev_fwd + 1: first task of each level
  int32_t* lptr_bwd = nullptr;
  int32_t* hptr_fwd = nullptr;  // nlev: end of the leading heavy rows of each level
  int32_t* hptr_bwd = nullptr;
  std::vector<int32_t> h_lptr_fwd, h_lptr_bwd;
  std::vector<int64_t> h_lwork_fwd, h_lwork_bwd;   // dependencies per level
  std::vector<int32_t> h_hptr_fwd, h_hptr_bwd;     // host copies of hptr
  // heavy rows split into dependency chunks for the grid solves, per direction and chunk size
  // (built on first use; device arrays owned by `mem`)
  struct ChunkPlan {
    void* chunk = nullptr;     // HeavyChunk array
    int32_t* cptr = nullptr;   // nlev + 1
    int max_slots = 0, max_rows = 0;
  };
  std::map<std::pair<int, int>, ChunkPlan> chunk_plans;   // (fwd, chunk size) -> plan
  // the leading levels [0, l_head) of the forward solve in task-position space: hpos[p * m + c]
  // is the position of dependency c of the row at position p (built on first use per l_head)
  struct HeadPlan {
    int32_t* hpos = nullptr;
    int rows = 0;
    bool usable = false;
  };
  std::map<int, HeadPlan> head_plans;
  // tiled solves (sptrsv_tile*_kernel): G tiles of R storage rows, each tile's rows by level,
  // the rows another tile depends on, and the ready flags of block solves (epoch per launch);
  // built on first use per (direction, G)
  struct TilePlan {
    int G = 0, R = 0;
    int32_t* ttask = nullptr;
    int32_t* toff = nullptr;
    uint8_t* exported = nullptr;
    int* flag = nullptr;
    int epoch = 0;
  };
  std::map<std::tuple<int, int, int>, TilePlan> tile_plans;   // (forward, G, first listed task)
  // staged products (spmv_*_staged_kernel): row blocks and the rows each reads, per (forward,
  // bytes per row); usable = false when some row reads more rows than shared memory holds
  struct HaloPlan {
    int nb = 0, ucap = 0;
    bool usable = false;
    int32_t* brow = nullptr;
    int32_t* uoff = nullptr;
    int32_t* ulist = nullptr;
    uint16_t* lidx = nullptr;
    uint16_t* lself = nullptr;
  };
  std::map<std::pair<int, int>, HaloPlan> halo_plans;
  // LRAC (Section 3.1.2): rank-k pivoted Cholesky factor of Sigma, built on first use
  // and dropped when the covariance parameters change
  Owned lrac_mem;
  int lrac_k = 0;
  double* L64 = nullptr;      // n x k, column-major over the storage rows
  float* L32 = nullptr;       // float copy, made on first float32 use
  int32_t* piv_s = nullptr;   // k pivots as storage rows
  int32_t* piv_v = nullptr;   // k pivots as Vecchia indices
};

struct State {
  Factor* f = nullptr;
  Ctx* ctx = nullptr;
  Owned mem;
  int lik = 0;
  double shape = 1.0;   // gamma shape (VL_LIK_GAMMA_LOG)
  int* d_seg_lik = nullptr;        // batches: likelihood and shape of every problem (device)
  double* d_seg_shape = nullptr;
  double* y = nullptr;     // storage order
  double* F = nullptr;
  double* b = nullptr;     // mode
  double* W = nullptr;
  int last_t = 0;
  std::vector<double> h_gammas;   // last SLQ gammas
  vl_stats mode_stats{};          // diagnostics of the Newton solve
};

// ----------------------------------------------------------------------------- helpers
// Whether memory that the CUDA driver describes as (type, device) may be handed straight to
// kernels running on device ctx_device: managed memory, or device memory of that device.
// Host-callable pure logic (tested on the CPU).
inline bool device_memory_usable(int type, int device, int ctx_device) {
  return type == cudaMemoryTypeManaged || (type == cudaMemoryTypeDevice && device == ctx_device);
}

vl_status cuda_fail(Ctx* c, cudaError_t e, const char* what);
vl_status fail(Ctx* c, vl_status s, const std::string& msg);
vl_status check_dev_status(Ctx* c, const char* what);   // syncs the stream
// Clears the device status (error code, row, abort flag), keeping the wait limit.
inline cudaError_t status_clear(Ctx* c) { return cudaMemsetAsync(c->dstatus, 0, kStatusClearBytes, c->stream); }
int resident_blocks(Ctx* c, const void* kernel, int block, size_t smem);

#define VL_CUDA(ctx, call)                                                 \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) return ::vl::cuda_fail((ctx), e_, #call);       \
  } while (0)

#define VL_TRY(call)                    \
  do {                                  \
    vl_status s_ = (call);              \
    if (s_ != VL_OK) return s_;         \
  } while (0)

// ----------------------------------------------------------------------------- launchers
// knn.cu
vl_status knn_prev_dev(Ctx* c, const double* locs_v, int64_t n, int m, int32_t* N_out);
vl_status knn_cross_dev(Ctx* c, const double* train, int64_t n, const double* test, int64_t np,
                        int m, int32_t* N_out);
vl_status morton_perm(Ctx* c, const double* locs, int64_t n, int32_t* perm_out);
vl_status bbox(Ctx* c, const double* locs, int64_t n, const double* extra, int64_t n_extra,
               double out[4]);

// graph.cu: storage order, ELL/transpose patterns, levels and task orders from
// the Vecchia-order neighbour table N_v and locations locs_v (both device).
vl_status build_graph_impl(Factor* f, const int32_t* N_v, const double* locs_v, const int32_t* order_dev);
vl_status refresh_transpose_values(Factor* f);

// lrac.cu: the rank-k pivoted Cholesky factor of Sigma for the LRAC preconditioner
// (f->L64, f->piv_*; rebuilt when k changes), and its float32 copy f->L32.
vl_status lrac_build(Factor* f, int k);
vl_status lrac_float(Factor* f);
void lrac_drop(Factor* f);

// factor.cu: A (rows x m) and D (rows) of the Vecchia rows; row_ids (optional)
// name rows in error messages.
vl_status factor_rows(Ctx* c, int64_t rows, int m, const double* self_locs, const double* ref_locs,
                      const int32_t* nbr, int cov, double sigma2, double rho, double nugget,
                      double* A, double* D, const int32_t* row_ids);

}  // namespace vl
