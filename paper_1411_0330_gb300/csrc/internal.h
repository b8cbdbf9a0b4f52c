// internal.h -- host-side declarations shared by the liblsh translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace lsh {

// Everything an operator pass needs, passed by value to the kernels.
//
// A launch covers S independent systems (one microstructure, one load each)
// that share the grid, the reference medium, the twiddles and the Gamma^h
// table.  Fields are stored system-major: [S][c][nz][ny][nx] (real) and
// [S][c][nz][ny][nxh] (half spectrum), so the rows of all systems are one
// contiguous range; each x-pass block works inside one system (RY divides the
// rows of a system) which keeps the per-system reductions block-aligned.
template <typename T> struct OpArgs {
  int nx, ny, nz, nxh, c;
  int hs;            // row stride of the half spectrum H (nxh rounded up to 4: 32-byte FP32 rows)
  int ts;            // row stride of the Gamma table (nxh rounded up to 8: 32-byte FP32 rows)
  long long V;       // voxels per system
  int S;             // systems in this launch
  int sys0;          // global index of system 0 of this launch
  int sys_per_ms;    // systems per microstructure (phase map index = (sys0 + s) / sys_per_ms)
  int rps;           // rows per system: c * nz * ny
  int bps;           // x-pass blocks per system: rps / RY
  int RY;            // rows per block in the x passes
  int TY, TZ;        // kx columns per block in the y / z passes
  int lsx, lsy, lsz; // shared-memory line strides (complex elements)
  Plan1D px, py, pz;
  const C2<T>* twx;
  const C2<T>* twy;
  const C2<T>* twz;
  const int* posx;   // frequency kx -> position after the x DIF
  C2<T>* H;          // half spectrum [S][c][nz][ny][hs] (kx < nxh used; y, z positions per kofy / kofz)
  const T* gtab;     // Gamma^h (internal basis, scaled by 1/V): blocks of 8 frequencies, see gamma_elem
  int ncoef;
  // local term M_beta = (A_beta - A0)^{-1}, diagonal in the internal basis
  const unsigned char* phase;  // [nbatch][V]
  const float* scale;          // [nbatch][V] or null
  int frac;                    // 1: scale holds the volume fraction of phase 1 (Eq. (def_ah))
  const unsigned char* act;    // per phase: 1 if A_phase != A0 (voxel in I0)
  int nphase;
  const T* mtab;               // per phase * c: diagonal of M (no scale field)
  const T* modtab;             // per phase * c: diagonal of A_phase (scale field)
  T ref[6];                    // diagonal of A0 (internal basis)
  const T* loads;              // [S][6] macroscopic load per system (internal basis)
  // Green operator computed in the z pass instead of read from gtab (truncated
  // operator, FP32): physics, grid lengths, signed-frequency tables, constants
  int onfly;                   // 1: compute Gamma^h_k on the fly
  int fdphase;                 // finite-difference operator: the table holds the real part
                               // u u^T / (u^T A0 u); components rotate by -/+ pi k_i / N_i around it
  int physics;
  const int* kofy;             // y position -> frequency
  const int* kofz;             // z position -> frequency
  T g0[6];                     // elastic: 1/(2 mu0 V), cb/V, 1/(3 K0 V), 1/(2 mu0 V); scalar: A0 diagonal
  T invV;
  // register-FFT passes (natural-order y / z frequencies) for lengths 16..256
  int yreg, zreg;
  // FP32 y and z passes through the Tensor Memory Accelerator (host pointers
  // to the maps)
  int ytma;           // 1: TMA y pass
  int ztma;           // 0: register z pass; 1..5: the variant of launch_zgamma_tma; 6: register, 4 columns;
                      // 7: persistent register z pass with staged prefetch; 8: register, 16 columns;
                      // 9: register, coefficients loaded when used; 10: pipelined TMA tiles on the
                      // ky-major spectrum (kernels_zpipe.cu); 11: the same on the plan N = R1 x 4
                      // with the 4-point DFTs and Gamma^h fused
  const CUtensorMap* tmy;
  const CUtensorMap* tmz;   // z boxes of 4 columns
  const CUtensorMap* tmz8;  // z boxes of 8 columns
  const CUtensorMap* tmz16; // z boxes of 16 columns
  const CUtensorMap* tmzp;  // ky-major spectrum, boxes of 8 columns (variant 10)
  const CUtensorMap* tmzq;  // Nyquist columns of the ky-major spectrum, boxes of 8 ky
  int* fault;  // set by a kernel whose bounded wait ran out
  int xreg;    // FP32 inverse x pass: 0 shared-memory stages, 1 register FFT, 2 register FFT persistent,
               // 3 register FFT in blocks of 128 threads
  int xfreg;   // 1: FP32 forward x pass on the register FFT (kernels_x.cu)
  // FP32 plane passes (kernels_plane.cu): x and y transforms of a z plane in one
  // kernel; the spectrum is then ky-major, H[S][c][ky][z][hs] (tlay = 1), and the
  // Nyquist column kx = nx/2 also lives in nq[S][c][z][ky]
  int plane;
  int tlay;
  C2<T>* nq;
  int l2pf;  // plane passes, input planes requested into L2 at a block's start: bit 0 the
             // forward pass's x, r, p; bit 1 the inverse pass's p and phase planes
};

// Thread-block sizes and tile shapes, chosen at setup for one system count.
struct LaunchCfg {
  int threads;
  int RY, TY, TZ, VEC;
  size_t smem_x, smem_y, smem_z;
  int grid_x, grid_yx, grid_yy, grid_zx, grid_zy, grid_zz;
  int ew_per_sys;  // blocks per system of the elementwise kernels
};

template <typename T>
void launch_xfwd(const OpArgs<T>& a, const LaunchCfg& L, int mode, const T* in, T* x, const T* r, T* p,
                 const SolverState* st, cudaStream_t s);
template <typename T>
void launch_yfft(const OpArgs<T>& a, const LaunchCfg& L, bool inv, const SolverState* st, cudaStream_t s);
template <typename T>
void launch_zgamma(const OpArgs<T>& a, const LaunchCfg& L, const SolverState* st, cudaStream_t s);
template <typename T>
void launch_xinv(const OpArgs<T>& a, const LaunchCfg& L, int mode, const T* xin, T* out, SolverState* st,
                 double* partials, cudaStream_t s);
template <typename T>
void launch_cg_update(T* r, const T* q, long long n, int S, SolverState* st, double* partials, int G, cudaStream_t s);
template <typename T>
void launch_cg_finalize(T* x, const T* p, long long n, int S, const SolverState* st, int G, cudaStream_t s);
template <typename T>
void launch_cg_begin(const T* r, long long n, int S, SolverState* st, double* partials, double tol,
                     const double* bb_given, int G, cudaStream_t s);
template <typename T>
void launch_fill_rhs(const OpArgs<T>& a, T* r, T* x, int G, cudaStream_t s);
template <typename T>
void launch_rotate(const T* in, T* out, long long V, int nsys, int to_internal, cudaStream_t s);
template <typename T>
void launch_comp_sums(const T* x, int c, long long V, int S, double* partials, int nblk, double* out, cudaStream_t s);
template <typename T>
void launch_gamma_table(const OpArgs<T>& a, int dim, int physics, int green, const double* ref_mandel,
                        const int* kofy, const int* kofz, cudaStream_t s, const double* a0full = nullptr,
                        const double* rot = nullptr);
template <typename T>
void launch_rotate_scalar(const T* in, T* out, long long V, int nsys, int d, const double* R, int to_internal,
                          cudaStream_t s);
void launch_d2f_begin(const double* r64, bool df_pairs, float* r32, float* x32, long long n, int S, SolverState* st,
                      double* partials, double tol, const unsigned char* active, int G, cudaStream_t s);
void launch_f2d_axpy(double* x64, const float* x32, long long n, cudaStream_t s);
void launch_scan_phase(const unsigned char* phase, long long V, int B, const unsigned char* act, int nphase,
                       SolverState* st, double* partials, int G, cudaStream_t s);
void launch_scale_grad(const double* tau_all, const double* W, const unsigned char* phase, const float* scale,
                       const double* modtab, const double* ref, int c, int elastic, long long V, int B,
                       double* grad, cudaStream_t s);

void launch_dot_finalize(SolverState* st, const double* partials, int nb, int S, cudaStream_t s);
void launch_basic_update(const OpArgs<double>& a, double* x, const double* r, const unsigned char* flags, int G,
                         cudaStream_t s);
void launch_minres_begin(SolverState* st, MinresScalars* ms, const double* rhs2, const double* bb, double tol, int S,
                         cudaStream_t s);
void launch_minres_step(double* x, double* r1, double* r2, double* q, double* wa, double* wb, long long n, int S,
                        SolverState* st, MinresScalars* ms, double* partials, int G, cudaStream_t s);
void launch_symmlq_begin(SymmlqScalars* sq, int S, cudaStream_t s);
void launch_symmlq_step(double* x, double* r1, double* r2, double* q, double* w, const double* b, long long n, int S,
                        SolverState* st, MinresScalars* ms, SymmlqScalars* sq, double* partials, int G,
                        cudaStream_t s);
template <typename T> void set_smem_attrs();
template <typename T> void set_smem_attrs_reg();
template <typename T> void launch_yfft_reg(const OpArgs<T>& a, bool inv, const SolverState* st, cudaStream_t s);
template <typename T> void launch_zgamma_reg(const OpArgs<T>& a, const SolverState* st, cudaStream_t s, int tz);
bool reg_length(int n);
void launch_yfft_tma(const OpArgs<float>& a, bool inv, const SolverState* st, cudaStream_t s);
bool encode_y_map(CUtensorMap* out, void* H, int hs, int ny, long long planes);
bool launch_zgamma_tma(const OpArgs<float>& a, int var, const SolverState* st, cudaStream_t s);
bool tma_z_variant_fits(const OpArgs<float>& a, int var);
bool launch_zgamma_regp(const OpArgs<float>& a, const SolverState* st, cudaStream_t s);
bool launch_zgamma_pipe(const OpArgs<float>& a, bool fused, const SolverState* st, cudaStream_t s);
bool encode_zpipe_maps(CUtensorMap* th, CUtensorMap* tq, void* H, void* NQ, int hs, int ny, int nz, int c,
                       long long nsys);
void zpipe_prepare();
int multiprocessors();
// double-float passes (kernels_df.cu); DF and DF2 come from df.cuh
struct DF;
struct DF2;
bool df_supported(const OpArgs<double>& a);
void launch_d2df(const double* in, DF* out, long long n, cudaStream_t s);
void launch_d2df_inplace(void* buf, long long n, cudaStream_t s);
void launch_df_x(const OpArgs<double>& a, const DF2* twx, int mode, const double* in, double* out, SolverState* st,
                 double* partials, cudaStream_t s);
void launch_df_z(const OpArgs<DF>& a, cudaStream_t s);
void df_prepare();
bool encode_z_map(CUtensorMap* out, void* H, int hs, int ny, int nz, int c, long long nsys, int tz);
void tma_prepare();
void launch_wait_probe(int* fault, unsigned long long limit_ns, cudaStream_t s);
bool launch_xinv_reg(const OpArgs<float>& a, int mode, const float* xin, float* out, SolverState* st,
                     double* partials, cudaStream_t s, bool persistent, bool small = false);
void xreg_prepare();
bool xinv_reg_fits(const OpArgs<float>& a);
bool launch_xfwd_reg(const OpArgs<float>& a, int mode, const float* in, float* x, const float* r, float* p,
                     const SolverState* st, cudaStream_t s);
bool xfwd_reg_fits(const OpArgs<float>& a);
bool plane_length(int n);
bool launch_xyfwd(const OpArgs<float>& a, int mode, const float* in, float* x, const float* r, float* p,
                  const SolverState* st, cudaStream_t s);
bool launch_xyinv(const OpArgs<float>& a, int mode, const float* xin, float* out, SolverState* st, double* partials,
                  cudaStream_t s);
void plane_prepare();

}  // namespace lsh
