// Host-side launchers of the CUDA-core kernels (simt.cu).
#pragma once

#include "kernels_simt.cuh"

namespace bcrown {

void launch_tables(int P, int H, const float* l, const float* u, Tables& t, uint8_t* code, int32_t* rank,
                   float* slope, float* icpt, int32_t* U, cudaStream_t s);
void launch_absw_m(const LayerGeom& g, const float* W, int P, int H, long long hoff_i, long long hoff_prev,
                   const float* u, const float* x_lo, const float* x_hi, int d0, float* wm, cudaStream_t s);
void launch_init_top(bool cert, const RowsCtx& c, int dtop, const bcrown_net* net, long long hoff_top, float* A,
                     float* cf, double* cd, double* E, cudaStream_t s);
void launch_relax(bool cert, const RowsCtx& c, int layer, int d, long long hoff, const float* Ain, float* Lam,
                  const float* bias, const float* alpha, int64_t n_alpha, const float* beta, int64_t n_beta, float* cf,
                  double* cd, double* E, const float* wm, double gamma, cudaStream_t s);
void launch_sgemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                  const float* bias, cudaStream_t s);
void launch_conv_bwd(int R, const LayerGeom& g, const float* Lam, const float* W, float* Ain, cudaStream_t s);
void launch_conv_fwd(int R, const LayerGeom& g, const float* h, const float* W, const float* bias, float* Z,
                     cudaStream_t s);
void launch_concretize(bool cert, const RowsCtx& c, int d0, const float* A0, const float* cf, const double* cd,
                       const double* E, float* lb, cudaStream_t s);
void launch_xstar(const RowsCtx& c, int d0, const float* A0, float* h0, cudaStream_t s);
void launch_fwd_epi(const RowsCtx& c, int layer, int d, long long hoff, float* Z, const float* Ai,
                    const float* alpha, int64_t n_alpha, float* dalpha, float* dbeta, int64_t n_beta,
                    cudaStream_t s);
void launch_adam(int R, int K, const BatchView& bt, const int32_t* U, int P, const float* lb_t, float* best_lb,
                 float* a_cur, float* a_best, const float* ga, float* ma, float* va, float* b_cur, float* b_best,
                 const float* gb, float* mb, float* vb, float lr_a, float lr_b, float beta1, float beta2, float eps,
                 float bc1, float bc2, int64_t n_alpha, int64_t n_beta, cudaStream_t s);
// As launch_adam with the alpha gradient and moments in BF16.
void launch_adam16(int R, int K, const BatchView& bt, const int32_t* U, int P, const float* lb_t, float* best_lb,
                   float* a_cur, float* a_best, const __nv_bfloat16* ga, __nv_bfloat16* ma, __nv_bfloat16* va,
                   float* b_cur, float* b_best, const float* gb, float* mb, float* vb, float lr_a, float lr_b,
                   float beta1, float beta2, float eps, float bc1, float bc2, int64_t n_alpha, int64_t n_beta,
                   cudaStream_t s);
void launch_codes(const RowsCtx& c, int layer, int d, long long hoff, int H, int8_t* out, cudaStream_t s);
void launch_split(const BatchView& bt, int K, const int32_t* U, int P, const uint8_t* pick_layer,
                  const uint32_t* pick_idx, const float* alpha, const float* beta, int32_t* c_prop, int32_t* c_off,
                  int32_t* c_cnt, int64_t* c_aoff, uint8_t* c_layer, uint32_t* c_idx, int8_t* c_sign,
                  float* c_alpha, float* c_beta, int* status, cudaStream_t s);
void launch_root_top(int q0, int Rc, int d_top, const float* b_top, float* Lam, float* cf, double* cd, double* E,
                     cudaStream_t s);
void launch_relax_root(bool cert, int Rc, int p, int H, int d, long long hoff, const float* l, const float* u,
                       const Tables& tb, int rule, float rule_value, const float* Ain, float* Lam, const float* bias,
                       float* cf, double* cd, double* E, const float* wm, double gamma, cudaStream_t s);
void launch_concretize_root(bool cert, int q0, int Rc, int p, int d0, int d_top, int H, long long hoff_top,
                            const float* x_lo, const float* x_hi, const float* A0, const float* cf, const double* cd,
                            const double* E, float* l, float* u, cudaStream_t s);
void launch_fill(float* p, long long n, float v, cudaStream_t s);
// FP32 implicit-GEMM convolutions (conv_f32.cu): the transposed convolution of conv layer i split
// into stride phases (backward), and the convolution plus bias (forward), for R rows.
constexpr int SCONV_MAX_K = 4096;   // terms per output the staged gather table holds
bool sconv_supported(const bcrown_net* net, int i);
int sconv_load(bcrown_net* net);   // builds the tables (at bcrown_load_net)
int sconv_bwd(bcrown_net* net, int i, int R, const float* Lam, float* Ain, cudaStream_t s);
int sconv_fwd(bcrown_net* net, int i, int R, const float* h, float* Z, const float* bias, cudaStream_t s);
void sconv_release(const bcrown_net* net);
void launch_relu(float* z, long long n, cudaStream_t s);
void launch_spec_out(int R, int K, int d, const float* h, const float* Wbar, const float* bbar, float* out,
                     cudaStream_t s);
void launch_f32_to_bf16(const float* src, __nv_bfloat16* dst, long long n, cudaStream_t s);
void launch_bf16_to_f32(const __nv_bfloat16* src, float* dst, long long n, cudaStream_t s);
void launch_copy_count(int P, int H, const int32_t* U, int32_t* out, cudaStream_t s);

}  // namespace bcrown
