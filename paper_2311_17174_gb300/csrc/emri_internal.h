// emri_internal.h -- host-side declarations shared by the libemri
// translation units (kernel launchers and normalised options).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace emri {

struct WalkerC;
struct Knot;
struct FdW;

// Largest grid y of a launch: the batched kernels put walkers (or
// sequences) on grid y, so a call processes at most this many per launch.
constexpr int kMaxGridY = 65535;

// Options after defaults and validation.
struct OptsN {
  int precision;   // 0 FP64, 1 mixed
  int n_max;
  int doppler;
  int pn_terms;
  int mode;        // 0 forward, 1 backward from LSO
  int ks;          // knot spacing (samples)
  double n_xi, omega_m, h0;
};

// FFT split of n = n1 * n2 (n2 = column length, n1 = row length).
struct FftPlan {
  int64_t n;
  int n1, n2;
  int log2n;
};
// n2 = 0: default split n2 = 2^min(10, log2(n)/2)
FftPlan make_fft_plan(int64_t n, int n2 = 0);

// Twiddle tables: ta[i] = exp(-2 pi i i/4096), i < 4096; tb[i] = exp(-2 pi i i/2^22), i < 1024.
struct Twiddles {
  double2* ta64;   // exp(-2 pi i k / 4096)
  double2* tb64;   // exp(-2 pi i k / 2^22), k < 1024
  float2* ta32;
  float2* tb32;
  double2* tc64;   // (cos, tan) of -2 pi k / 4096, |cos| >= 2^-60
  float2* tt32;    // stage twiddles: tt32[M/2 + k] = exp(-2 pi i k / M), M = 2..4096, k < M/2
};

void launch_twiddle_init(Twiddles t, cudaStream_t s);

// Bessel series tables: c[m * kBesselTerms + k] = (-1)^k m!/(k! (m+k)!),
// f[m] = 1/m!, m < kBesselOrders
constexpr int kBesselOrders = 35;
constexpr int kBesselTerms = 48;
struct BesselTab {
  double* c64;
  float* c32;
  double* f64;
  float* f32;
};
// fills the tables from the host (synchronous); 0 on success
int upload_bessel_tables(const BesselTab& t);
// the FP64 waveform kernel's exp(2 pi i k/512) table on the current device; 0 on success
int upload_exp512();

void launch_prologue(const double* theta, int64_t ld, int w, int64_t n, double dt, const OptsN& o,
                     const double* gl, WalkerC* out, cudaStream_t s);
// tab[w][n1] = exp(-2 pi i frac(n2 k1 r)), rtab[w][n2] = exp(-2 pi i frac(k2 r))
void launch_delay_table(const WalkerC* wc, int w, int n1, int n2, bool fp32, void* tab, void* rtab, cudaStream_t s);
void launch_prologue_export(const WalkerC* wc, int w, double* out, cudaStream_t s);
// frequency-dependent propagation records fd[w] from theta and coef[qm+qt][ldc]
void launch_fdprop(const double* theta, int64_t ld, int w, int64_t n, double dt, const OptsN& o, int qm, int qt,
                   double fstar, const double* coef, int64_t ldc, FdW* fd, cudaStream_t s);

// orbit: knots[w][nk+1], nk = n / ks
// mcpi_tab: Chebyshev-Picard tables (qn then qk), required
void launch_orbit(WalkerC* wc, int w, int64_t n, double dt, double t0, const OptsN& o, Knot* knots,
                  const double* mcpi_tab, cudaStream_t s);

// waveform: z[w][n] (double2 or float2); unit_scale multiplies by mu_s c (cm units)
// lisa: per-tile phibar table [n/256][8] (launch_lisa_tiles); ivs: mixed
// interval records [w][n/ks] (launch_intervals_mixed; unused for FP64)
void launch_wave(const Knot* knots, const WalkerC* wc, int w, int64_t n, double dt, double t0,
                 const OptsN& o, void* z, bool unit_scale, const BesselTab& bt, const double* lisa, const void* ivs,
                 cudaStream_t s);
void launch_intervals_mixed(const Knot* knots, int w, int64_t n, int ks, double dt, void* ivs, cudaStream_t s);
void launch_lisa_tiles(int64_t n, double t0, double dt, double* tab, cudaStream_t s);
constexpr size_t kIvMBytes = 104;

// FFT pass 1 (columns, in place, with the inter-pass twiddle); sign -1 forward, +1 inverse
void launch_fft_pass1(void* z, int batch, const FftPlan& p, bool fp32, int sign, const Twiddles& t,
                      cudaStream_t s);
// FFT pass 2 to natural order into out (out-of-place)
void launch_fft_pass2_store(const void* y, void* out, int batch, const FftPlan& p, bool fp32, int sign,
                            const Twiddles& t, cudaStream_t s);
// FFT pass 2 fused with the weighted inner products; partial[w][n2] = (dh, hh)
void launch_fft_pass2_ip(const void* y, int w, const FftPlan& p, bool fp32, const Twiddles& t,
                         const WalkerC* wc, const void* delay_tab, const void* row_tab, const void* data_perm,
                         const void* wt_perm, double2* partial, cudaStream_t s, const FdW* fd = nullptr);
// per-walker fixed-order reduction of the partials and lnL
// dh_scale / hh_scale undo the dataset's FP32 scaling (1 for FP64)
void launch_finalize(const double2* partial, int n2, const WalkerC* wc, int w, double dh_scale, double hh_scale,
                     double* lnl, double* dh, double* hh, uint32_t* status, cudaStream_t s);
void fft_set_smem_limits();

// dataset preparation: the weighted conjugate spectrum g = w conj(D) and
// the weights w in the pass-2 order (k2-major), plus FP32 copies scaled by
// d_scale w_scale and w_scale
void launch_dataset_permute(const double2* d_nat, const double* w_nat, const FftPlan& p, double2* g_perm,
                            double* w_perm, float2* g_perm32, float* w_perm32, double d_scale,
                            double w_scale, cudaStream_t s);
void launch_weights(const double* psd, int64_t n, double dt, double fmin, double fmax, double* w,
                    cudaStream_t s);
void launch_pack_time_series(const double* d2, int64_t n, double2* z, cudaStream_t s);
void launch_inner_dd(const double2* d, const double* w, int64_t n, double* out, cudaStream_t s);

}  // namespace emri
