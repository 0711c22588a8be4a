// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/bcrown.h"

namespace bcrown {

// ----------------------------------------------------------------------------------------
// Error handling
// ----------------------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

#define BC_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t _e = (call);                                                             \
    if (_e != cudaSuccess)                                                               \
      return ::bcrown::fail(BCROWN_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
  } while (0)

#define BC_CHECK(x)                        \
  do {                                     \
    int _s = (x);                          \
    if (_s != BCROWN_OK) return _s;        \
  } while (0)

// ----------------------------------------------------------------------------------------
// Network
// ----------------------------------------------------------------------------------------
struct LayerDev {
  int kind;
  int in_c, in_h, in_w, out_c, out_h, out_w, k, stride, pad;
  int d_in, d_out;
  float* W = nullptr;           // fc [d_out][d_in]; conv [out_c][in_c][k][k]
  float* Wt = nullptr;          // fc [d_in][d_out]
  float* b = nullptr;           // [d_out], conv bias expanded per position
  __nv_bfloat16* Wbf = nullptr;  // fc [d_out][d_in]   (rows = N, K-major for the forward)
  __nv_bfloat16* Wtbf = nullptr; // fc [d_in][d_out]   (rows = N, K-major for the backward)
  int terms_bwd = 0;             // max terms in one backward dot product
  int terms_fwd = 0;             // max terms in one forward dot product
};

// Geometry of one linear layer, passed by value to kernels.
struct LayerGeom {
  int kind;
  int in_c, in_h, in_w, out_c, out_h, out_w, k, stride, pad;
  int d_in, d_out;
};

inline LayerGeom geom_of(const LayerDev& l) {
  return LayerGeom{l.kind, l.in_c, l.in_h, l.in_w, l.out_c, l.out_h, l.out_w, l.k, l.stride, l.pad, l.d_in, l.d_out};
}

struct Workspace {
  void* ptr = nullptr;
  size_t size = 0;
};

}  // namespace bcrown

struct bcrown_net {
  int L = 0;                          // number of linear layers
  int K = 0;                          // number of specs
  std::vector<bcrown::LayerDev> ly;   // ly[i-1] holds paper layer i
  std::vector<int> d;                 // d[0..L]
  std::vector<long long> hoff;        // hidden offsets, hoff[i-1] = first neuron of layer i
  int H = 0;
  int max_hidden = 0;
  int max_width = 0;                  // max over d[0..L-1]
  float* Wbar = nullptr;              // [K][d_{L-1}]
  float* bbar = nullptr;              // [K]
  double* bbar_rd = nullptr;          // [K], a lower bound of the exact C b^(L)
  float* Wbar_err = nullptr;          // [K][d_{L-1}], bound on |Wbar - exact C W^(L)|
  __nv_bfloat16* Wbar_bf = nullptr;   // [K][d_{L-1}]
  int* status = nullptr;              // device status word
  // BF16 launch configuration: the caller's choice (bcrown_set_launch; path 0 = the built-in
  // order) and the tuner's per row-count bucket (bcrown_autotune), looked up on every call
  struct Launch {
    int path = 0;
    int grid_per_sm = 0;
  };
  Launch launch_set;
  std::vector<std::pair<int, Launch>> tuned;   // (bucket = ceil(log2 rows), choice)
  Launch launch_now;                           // the configuration of the call in progress
  bcrown::Workspace ws;
  std::mutex mu;
  // timing hook (bcrown_profile)
  bool prof_on = false;
  struct ProfRec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> evpool;
};

namespace bcrown {

// ----------------------------------------------------------------------------------------
// Device-side views passed by value to kernels
// ----------------------------------------------------------------------------------------
struct BatchView {
  int B;
  const int32_t* prop_of;
  const int32_t* split_off;
  const int32_t* split_cnt;
  const uint8_t* split_layer;
  const uint32_t* split_idx;
  const int8_t* split_sign;
  const int64_t* alpha_off;
};

struct Tables {            // per property, per hidden neuron (derived from l, u each call)
  int P, H;
  const uint8_t* code;     // 0 inactive, 1 active, 2 unstable
  const int32_t* rank;     // rank among unstable neurons (layer-major), -1 if stable
  const float* slope;      // u/(u-l)     (unstable)
  const float* icpt;       // -u*l/(u-l)  (unstable)
  const int32_t* U;        // [P] number of unstable neurons
};

enum : uint8_t { CODE_INACTIVE = 0, CODE_ACTIVE = 1, CODE_UNSTABLE = 2, CODE_SPLIT_POS = 3, CODE_SPLIT_NEG = 4 };

void* ws_get(bcrown_net* net, size_t bytes, int* status);   // grow-only workspace

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// A bump allocator over the workspace.
struct Arena {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t n) {
    T* p = reinterpret_cast<T*>(base + off);
    off += align_up(n * sizeof(T));
    return p;
  }
};

// Records an event pair around the kernels issued in its scope when profiling is on.
struct ProfScope {
  bcrown_net* net;
  int idx = -1;
  cudaStream_t s;
  ProfScope(bcrown_net* n, int cls, cudaStream_t st);
  ~ProfScope();
};

inline int grid1d(long long n, int block) { return (int)((n + block - 1) / block); }

}  // namespace bcrown
