// Internal declarations of the CG-DIR CUDA library (sm_103a).  Kernels live
// in kernels_*.cu, each with a host launcher declared here; runtime.cu owns
// the contexts, the pyramid and the C ABI of include/cgdir.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "cgdir.h"
#include "imgtype.cuh"

namespace cgdir {

constexpr int kMaxMasks = CGDIR_MAX_MASKS;
constexpr int kMaxRadius = 6;            // Gaussian radius ceil(3 sigma), sigma <= 2

struct Grid {
    int nx, ny, nz;
    __host__ __device__ size_t n() const { return (size_t)nx * ny * nz; }
};

__host__ __device__ __forceinline__ int clampi(int v, int lo, int hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}
__host__ __device__ __forceinline__ size_t vox(int x, int y, int z, int nx, int ny) {
    return ((size_t)z * ny + y) * nx + x;
}

// Trilinear corner set of a continuous position: coordinates clamped to
// [0, n-1], lower corner floor(p), upper corner clamped, weight p - floor(p).
struct Corners {
    int x0, x1, y0, y1, z0, z1;
    float wx, wy, wz;
};
__device__ __forceinline__ Corners corners(float px, float py, float pz, int nx, int ny, int nz) {
    Corners c;
    px = fminf(fmaxf(px, 0.f), (float)(nx - 1));
    py = fminf(fmaxf(py, 0.f), (float)(ny - 1));
    pz = fminf(fmaxf(pz, 0.f), (float)(nz - 1));
    float fx = floorf(px), fy = floorf(py), fz = floorf(pz);
    c.x0 = (int)fx; c.y0 = (int)fy; c.z0 = (int)fz;
    c.x1 = min(c.x0 + 1, nx - 1); c.y1 = min(c.y0 + 1, ny - 1); c.z1 = min(c.z0 + 1, nz - 1);
    c.wx = px - fx; c.wy = py - fy; c.wz = pz - fz;
    return c;
}

// Gaussian taps for kernel 1: exp(-j^2 / (2 sigma^2)) / sum, j in [-R, R].
struct Taps {
    int r;
    float w[2 * kMaxRadius + 1];
};
int gauss_radius(float sigma);
Taps gauss_taps(float sigma);

// Per-block partial sums of the stopping metric: {sum (I0~ - T0)^2 over the
// UROI, UROI count, max |du|}, FP64, written by the force / metric kernels.
constexpr int kPartialStride = 4;

// Device-side state of one level's stopping logic, updated by the reduction.
struct LevelState {
    double *hist;       // [hist_cap]
    int *hist_len;
    int *iters_run;
    int *stop_reason;
    int *stop_flag;
    int hist_cap;
};

// The reduction and stop test of one iteration, run by the last CTA of the
// kernel that wrote the per-CTA partials (the CTA that brings `done` to the
// grid size); it sums the partials in a fixed order, so the result does not
// depend on which CTA finishes last.
struct FinishArgs {
    unsigned *done;      // completion counter, 0 before the launch (reset by the last CTA);
                         // null = no fused reduction
    LevelState st;
    int n, cap, stop_mode;
    double eps;
    double *stats_out;   // optional {sum, count, max}
};

struct ForceArgs {
    const void *I0, *T0;      // images of type img_dtype (CGDIR_F32 / F16 / BF16)
    int img_dtype;
    const uint8_t *mbits, *sbits, *uroi;
    const void *mtex;         // moving texels (see imgtype.cuh); used by the TMA kernel
                              // when the contour terms are on (null otherwise)
    const float *u;
    float *du, *warped;
    double *partial;          // [gridDim.x*gridDim.y*gridDim.z][kPartialStride] or null
    const int *stop_flag;     // kernels return at once when *stop_flag != 0 (may be null)
    int nx, ny, nz;
    int k, contour;
    float offset;
    float lambda[kMaxMasks];
    float half_sign[kMaxMasks];   // s_i / 2
    FinishArgs fin;               // fused reduction (fin.done null = none)
    // Two-pass force (used when wfield is set and the volume has < 2^31
    // voxels): pass 1 writes I0~ to wfield, the corners' mask AND << 8 | OR
    // to wstate and, where the corners disagree on bit j, P_j to
    // pfield[j][N]; pass 2 takes the stencils from them.
    float *wfield;
    uint16_t *wstate;
    float *pfield;
    int pass2_width;              // voxels per thread in pass 2: 1 or 2 (at most), 0 = the
                                  // widest the shape and the fields' alignment allow
    int skip_warp;                // 1: pass 1's outputs are already current for u (the fused
                                  // smoothing + warp kernel wrote them): launch pass 2 only
};

// One whole pyramid level (all iterations of Algorithm A) in one cooperative
// launch: every CTA is resident, phases are separated by bounded grid
// barriers (see kernels_force.cu, k_level_coop).  For small levels, whose
// per-iteration kernels are too short to fill the GPU.
struct LevelCoopArgs {
    ForceArgs f;                  // images, masks, texels, structure terms, u (in/out), du,
                                  // two-pass scratch (wfield / wstate / pfield), UROI;
                                  // f.fin.st is the level's stop state; f.fin.cap / stop_mode / eps
    float *tmp1, *tmp2, *ub;      // 3N floats each
    Taps tf, td;                  // Gaussian taps of du and of u
    int compose_mode;
    unsigned long long *sums;     // [2][4] zeroed before the launch
    unsigned *bar;                // [2] grid-barrier counter and generation, zeroed before the launch
    int *err;                     // set to 1 if a barrier wait ran out
};
// CTAs of the cooperative level kernel for this level (0: cannot run it).
int level_coop_grid(int nx, int ny, int nz, bool contour, int img_dtype);
cudaError_t launch_level_coop(const LevelCoopArgs &p, int grid, cudaStream_t s);

// Image type of pyramid level l (0 = coarsest) of L when the registration
// stores its images as `storage`: the finest level (the input resolution,
// 7/8 of the pyramid's voxels) in that type, the coarser levels in float32.
// The box mean lowers the image noise by sqrt(8) per level, so a 16-bit
// rounding of a restricted image weighs 2.8x, 8x, ... more against it than
// at the finest level; the coarse levels' DVF, prolongated, then carries
// that error to the end.
inline int level_storage(int storage, int l, int L) { return l == L - 1 ? storage : CGDIR_F32; }

// Bytes of the two-pass force scratch for n voxels and k structures.
inline size_t force_scratch_bytes(size_t n, int k) {
    return n * 4 + ((n * 2 + 255) / 256) * 256 + (size_t)k * n * 4 + 512;
}
// Point the two-pass scratch fields of `a` into `scratch` (n voxels).
inline void force_scratch_assign(ForceArgs &a, void *scratch, size_t n) {
    char *p = static_cast<char *>(scratch);
    a.wfield = reinterpret_cast<float *>(p);
    a.wstate = reinterpret_cast<uint16_t *>(p + ((n * 4 + 255) / 256) * 256);
    a.pfield = reinterpret_cast<float *>(p + ((n * 4 + 255) / 256) * 256 + ((n * 2 + 255) / 256) * 256);
}

// Process-wide count of kernels launched by this library (instrumentation).
void note_launch(unsigned n = 1);

// Raise a kernel's dynamic shared-memory limit to `bytes` on the current
// device (the runtime call is made once per kernel, device and size).
cudaError_t ensure_smem(const void *func, size_t bytes);

// z-chunk length for a z-marching kernel with `xy_ctas` CTAs per chunk so the
// grid covers about `waves` x (resident CTAs per SM x SM count).
int pick_zchunk(int nz, long xy_ctas, int resident_per_sm, int waves);
int sm_count();

// ---- launchers (return the launch status; all async on `s`) ------------
// err: device word for bounded-wait timeouts; nullptr selects the plain kernel.
cudaError_t launch_force(const ForceArgs &a, int zchunk, int *nblocks_out, cudaStream_t s,
                         int *err = nullptr);
size_t force_partial_count(int nx, int ny, int nz, int zchunk);
int force_default_zchunk(int nx, int ny, int nz);
cudaError_t launch_metric(const void *I0, const void *T0, int img_dtype, const float *u,
                          const uint8_t *uroi, int nx, int ny, int nz, double *partial,
                          const int *stop_flag, int *nblocks_out, cudaStream_t s,
                          const FinishArgs *fin = nullptr);
size_t metric_partial_count(int nx, int ny, int nz);
cudaError_t launch_finalize(const double *partial, int nblocks, LevelState st, int n, int cap,
                            int stop_mode, double eps, double *stats_out, cudaStream_t s);

// Smoothing kernel variants: the TMA z-march (large volumes), the 3-D
// shared-memory tile (small volumes), the split xy + z kernels (needs a 3N
// scratch field; with the composite update fused into the z pass), the
// fused iteration schedule (3-D tiles of all three components with the
// composite update fused into the du pass and the next warp into the u
// pass; a standalone smoothing takes the tile kernel), or chosen by size.
// SMOOTH_MARCH takes the wide-tile z-march (64 x 16 tiles, nx % 8 == 0, R <= 4)
// where it applies, else the 32 x 16 one; SMOOTH_MARCH_NARROW always the
// 32 x 16 one (same bits; a context setting for comparisons, never tuned).
enum { SMOOTH_AUTO = 0, SMOOTH_MARCH = 1, SMOOTH_TILE = 2, SMOOTH_SPLIT = 3, SMOOTH_FUSED = 4,
       SMOOTH_MARCH_NARROW = 5 };
static_assert(SMOOTH_MARCH == CGDIR_SMOOTH_MARCH && SMOOTH_TILE == CGDIR_SMOOTH_TILE &&
                  SMOOTH_SPLIT == CGDIR_SMOOTH_SPLIT && SMOOTH_FUSED == CGDIR_SMOOTH_FUSED &&
                  SMOOTH_MARCH_NARROW == CGDIR_SMOOTH_MARCH32,
              "internal smoothing variants are the public tuning codes");
int smooth_auto_variant(int nx, int ny, int nz);
// Kernel choice for one smoothing launch: variant and (z-march) z chunk, 0 = default.
struct SmoothChoice {
    int variant = SMOOTH_AUTO;
    int zchunk = 0;
    int ctas_per_sm = 0;          // at most this many wide z-march CTAs per SM (0: no cap)
};
int smooth_default_zchunk(int nx, int ny, int nz, int ncomp);
// err: device word set to 1 if a bounded wait inside the kernel ran out;
// nullptr selects the plain-load kernel (no waits).
cudaError_t launch_smooth(const float *in, int ncomp, float sigma, int nx, int ny, int nz,
                          float *out, const int *stop_flag, cudaStream_t s, int *err = nullptr,
                          SmoothChoice ch = SmoothChoice(), float *scratch = nullptr);
cudaError_t launch_compose(const float *u, const float *du, int mode, int nx, int ny, int nz,
                           float *out, const int *stop_flag, cudaStream_t s);
// Algorithm A steps 2 + 3: out = G(du) + u(x + G(du)) (or u + G(du)).  By
// default G(du) goes to tmp (3N floats) and a composite-update kernel
// follows; one_pass fuses both into one TMA kernel over all three
// components (fewer bytes, but register-bound and slower on GB300).
cudaError_t launch_smooth_compose(const float *du, const float *u, int mode, float sigma, int nx, int ny,
                                  int nz, float *out, float *tmp, const int *stop_flag, cudaStream_t s,
                                  int *err, bool one_pass = false, SmoothChoice ch = SmoothChoice());
cudaError_t launch_warp(const float *f, const float *u, int nx, int ny, int nz, float *out,
                        cudaStream_t s);

// Fused iteration schedule (kernels_fused.cu), 8 x 8 x 8 tiles of all three
// components with their Gaussian halo in shared memory:
//   out = G(du) + u(x + G(du))  (or u + G(du))       Algorithm A steps 2-3
// err: device word set to 1 if the bounded wait for the tile's TMA copy ran out.
cudaError_t launch_fused_smooth_compose(const float *du, const float *u, int mode, float sigma, int nx, int ny,
                                        int nz, float *out, const int *stop_flag, int *err, cudaStream_t s);
//   u = G(in), then the first force pass at the new u into a's two-pass
//   scratch (a.wfield / wstate / pfield; a.u is not read)     step 4 + the
//   next iteration's warp
cudaError_t launch_fused_smooth_warp(const float *in, float sigma, float *u, const ForceArgs &a, int *err,
                                     cudaStream_t s);
// Whether the fused schedule can run for this force configuration (the
// two-pass force with 32-bit indexing).
bool fused_schedule_ok(const ForceArgs &a);

cudaError_t launch_pack_masks(const uint8_t *const *masks, int k, size_t n, uint8_t *bits,
                              cudaStream_t s);
cudaError_t launch_restrict_image(const void *in, int dtype, int nx, int ny, int nz, void *out,
                                  cudaStream_t s);
// The same from an in_dtype level into an out_dtype level.
cudaError_t launch_restrict_image(const void *in, int in_dtype, int nx, int ny, int nz, void *out, int out_dtype,
                                  cudaStream_t s);
cudaError_t launch_restrict_bits(const uint8_t *in, int nx, int ny, int nz, uint8_t *out,
                                 cudaStream_t s);
cudaError_t launch_prolong(const float *uc, int cx, int cy, int cz, int nx, int ny, int nz,
                           float *uf, cudaStream_t s);
cudaError_t launch_uroi(const uint8_t *sbits, int k, int nx, int ny, int nz, const double *spacing,
                        double margin, uint8_t *scratch, uint8_t *out, cudaStream_t s);
size_t uroi_scratch_bytes(size_t n);
cudaError_t launch_sign_sums(const void *T0, int dtype, const uint8_t *sbits, int k, int nx, int ny, int nz,
                             uint8_t *tmp_a, uint8_t *tmp_b, double *partial,
                             double *sums /* [k][4] */, cudaStream_t s);
size_t sign_partial_rows(size_t n);
// Convert n image values from in_dtype to out_dtype (round to nearest even).
cudaError_t launch_convert_image(const void *in, int in_dtype, size_t n, void *out, int out_dtype,
                                 cudaStream_t s);
// Interleave the moving image with its mask bits into texels (imgtype.cuh).
cudaError_t launch_make_texels(const void *I0, int dtype, const uint8_t *bits, size_t n, void *tex,
                               cudaStream_t s);

}  // namespace cgdir
