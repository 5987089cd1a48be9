/*
 * cmb3d.h -- C ABI of the GB300 (sm_103a) library for simulating partial-sky
 * CMB temperature maps with 3-D FFTs (the "3-D Fourier method" of Giner
 * Mascarell & Bunn, "Simulating Partial Sky Cosmic Microwave Background Maps
 * with 3D Fast Fourier Transforms").
 *
 * The method (paper Sec. II): given a 3-D power spectrum P_inf(k) whose
 * correlation function matches the angular one of a target C_l (Sec. II.A-B),
 * fill a periodic N^3 box of side L with complex normal Fourier coefficients of
 * variance P_box(|k|) = P_inf(|k|) (2 pi / L)^3 (Eq. 2.11 for a cubic box),
 * inverse-FFT it (Sec. II.D.1), and sample the field by interpolation at the
 * pixel positions r * n_hat on a sphere of radius r centred in the box.
 *
 * Conventions used by every call:
 *   - Every function returns CMB3D_OK (0) or a negative status and never throws
 *     or aborts across the ABI.  Output buffers are undefined after an error.
 *     cmb3d_strerror() names a status; cmb3d_error_detail() returns a message
 *     about the most recent error on the calling thread.
 *   - A plan is not thread-safe.  Work is enqueued on the CUDA stream passed
 *     as `stream` (a cudaStream_t; NULL = legacy default stream); ordering and
 *     synchronisation are the caller's, except where a call says it
 *     synchronises.
 *   - "device pointer" means memory of the plan's device (the device current
 *     when cmb3d_plan was called); "host pointer" means ordinary host memory.
 *     The plan copies every input array it is given; the caller keeps
 *     ownership of all buffers it passes.
 *   - Box layout: grid point (x, y, z) sits at (x, y, z) * L / N, periodic; the
 *     sphere centre is the box centre, so pixel n_hat maps to grid coordinates
 *     u = (r n_hat + L/2) / (L/N).  The real field is stored float[z][y][x].
 *   - Randomness: realization `seed` is a pure function of (plan, spectrum,
 *     seed); Fourier mode (m_x, m_y, m_z) draws from the Philox4x32-10 counter
 *     (m_x, m_y, m_z mod N/2, 0) with key (seed low 32 bits, seed high 32
 *     bits), words (0,1) for m_z < N/2 and (2,3) otherwise.
 */
#ifndef CMB3D_H
#define CMB3D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cmb3d_plan_s* cmb3d_plan_t;

/* Status codes. */
enum {
  CMB3D_OK = 0,
  CMB3D_EINVAL = -1,        /* bad argument (null pointer, size, range)            */
  CMB3D_ENOMEM = -2,        /* host or device allocation failed                     */
  CMB3D_ECUDA = -3,         /* a CUDA runtime call or kernel launch failed          */
  CMB3D_ENOSPEC = -4,       /* realization requested before cmb3d_set_spectrum      */
  CMB3D_ETIMEOUT = -5,      /* a bounded device-side wait gave up                   */
  CMB3D_EUNSUPPORTED = -6   /* valid request outside what this build supports       */
};

/* Interpolation of the box field at the pixels (paper Sec. II.D.1). */
enum {
  CMB3D_TRILINEAR = 1,      /* 2x2x2 taps, weights (1-t, t)                          */
  CMB3D_TRICUBIC = 3        /* 4x4x4 taps, Keys cubic convolution a = -1/2          */
};

/* Plan flags (bitwise OR). */
enum {
  CMB3D_FLAG_NONE = 0u,
  CMB3D_FLAG_NO_SORT = 1u << 0,       /* gather in the caller's pixel order          */
  CMB3D_FLAG_ALLOW_WRAP = 1u << 1,    /* permit L <= 2r (the sphere wraps around)    */
  CMB3D_FLAG_STAGE_TIMING = 1u << 2,  /* record CUDA events around every kernel      */
  CMB3D_FLAG_THREE_PASS = 1u << 3,    /* only separate y and x passes                  */
  CMB3D_FLAG_FUSED_YX = 1u << 4,      /* the fused y+x pass where it exists
                                         (128 <= N <= 1024)                            */
  CMB3D_FLAG_AUTOTUNE = 1u << 5,      /* at the first realization, time every kernel
                                         shape of this N and keep the fastest (cached
                                         per device and N for the process)            */
  CMB3D_FLAG_FP16_GEMM = 1u << 6,     /* y pass with its radix-16 stages as split-FP16
                                         (hi+lo) DFT-GEMMs on the tensor cores, FP32
                                         accumulation (N = 256, 512, 1024; else
                                         CMB3D_EUNSUPPORTED); tolerance 1e-3 of rms    */
  CMB3D_FLAG_NO_PRUNE = 1u << 7,      /* sky maps transform the whole box: by default
                                         (N >= 128) the y pass covers only the z-planes
                                         and stores only the (z, y) rows, and the x pass
                                         only the rows, that the pixels' interpolation
                                         stencils read; the maps are identical          */
  CMB3D_FLAG_PIPELINE = 1u << 8,      /* a second box (4 N^3 more bytes) and two
                                         internal streams: the draw of a sky map
                                         overlaps the passes and gather of the previous
                                         map of the plan.  Stream semantics are kept:
                                         the map's kernels run after the caller's stream
                                         at the call, and the caller's stream waits for
                                         the map.  Maps are identical                   */
  CMB3D_FLAG_FUSED_XG = 1u << 9       /* sky maps run the x pass and the gather as one
                                         kernel: pixels are grouped by 8 x 8 tiles of
                                         (z, y) base cells, each tile's block forms the
                                         real rows its stencils read in shared memory
                                         (only the needed x columns) and interpolates
                                         from there; the real field is never written.
                                         32 <= N <= 2048 (no effect below); 20 more
                                         bytes per pixel.  Maps equal those of the
                                         separate passes with the x shape of the same
                                         radix (x variant 1 at N = 1024; 0 else) bit
                                         for bit.  Batches keep the separate
                                         passes; cmb3d_realize_field is unchanged      */
};

/* Spectrum kinds for cmb3d_set_spectrum. */
enum {
  CMB3D_SPEC_PK = 0,        /* x = k nodes, y = P_inf(k) at the nodes               */
  CMB3D_SPEC_CL = 1         /* x = multipoles l, y = C_l (inverted to P_inf(k))     */
};

/* Kernel stages of one realization, for cmb3d_stage_times(). */
enum {
  CMB3D_STAGE_DRAW_ZFFT = 0,   /* Philox draw x sqrt(P_box), Hermitian, 1-D FFT along z */
  CMB3D_STAGE_YFFT = 1,        /* 1-D FFT along y                                       */
  CMB3D_STAGE_XC2R = 2,        /* 1-D complex-to-real FFT along x                       */
  CMB3D_STAGE_GATHER = 3,      /* interpolation at the pixels                           */
  CMB3D_STAGE_YX_FUSED = 4,    /* y and x passes fused per z-plane (cluster, via L2)    */
  CMB3D_NUM_STAGES = 5
};

/*
 * Create a plan for an N^3 box of side L sampled at npix pixels on the sphere
 * of radius r (paper Sec. II.C on the box, Sec. II.D.1 on sampling).
 *
 *   out      [out] receives the new plan (set to NULL on error).
 *   N        points per axis; a power of two with 8 <= N <= 2048, else
 *            CMB3D_EUNSUPPORTED.
 *   L, r     box side and sphere radius, finite and > 0; L > 2r is required
 *            unless flags has CMB3D_FLAG_ALLOW_WRAP (CMB3D_EINVAL).
 *   pix_xyz  host pointer, npix x 3 doubles (x, y, z of each unit vector,
 *            row-major); may be NULL when npix == 0.  Copied.
 *   npix     number of pixels, 0 <= npix < 2^31.
 *   interp   CMB3D_TRILINEAR or CMB3D_TRICUBIC.
 *   flags    CMB3D_FLAG_* bits.
 * Pixel positions are mapped once, in IEEE double precision evaluated as
 * u = (r * n + 0.5 * L) / (L / N) with no fused multiply-add: the base cell
 * floor(u) mod N is kept exactly and the fraction u - floor(u) is rounded to
 * binary32.  Allocates the plan's device memory: 4 N^3 bytes for the box plus
 * 20 bytes per pixel plus small tables.
 */
int cmb3d_plan(cmb3d_plan_t* out, int N, double L, double r,
               const double* pix_xyz, int64_t npix, int interp, uint32_t flags);

/*
 * Create a plan for the 2-D Fourier method (paper Sec. II.D.2): the box is
 * simulated in Fourier space along x and y and in real space along z, on the
 * h layers that hold the cap only.  For each (m_x, m_y) the h values are
 * correlated Gaussians, S c with S the symmetric square root of the h x h
 * covariance Gamma_ij = xi(|i - j| dp) along z (xi: the transform of the box
 * spectrum along m_z over the z-period M dp) and c complex normals; a 2-D
 * inverse FFT per layer gives the real layers, which are sampled at the
 * pixels as in the 3-D method.  The cap is not required to fit in a cube:
 * x and y are periodic with side L, z is not.
 *
 *   N        points along x and y; a power of two with 16 <= N <= 2048.
 *   M        z-period in grid steps (the never-built N x N x M box of
 *            Sec. II.C), 1 <= M <= 65536.
 *   h        simulated layers, 1 <= h <= 32 and h <= N (else
 *            CMB3D_EUNSUPPORTED); layer j sits at z = z0 + j L/N.
 *   L, r     side of the box in x and y, sphere radius; finite and > 0.
 *   z0       height of layer 0, finite.
 *   pix_xyz, npix, interp as for cmb3d_plan.  A pixel maps to
 *            u = ((r n_x + L/2), (r n_y + L/2), (r n_z - z0)) / (L/N) in IEEE
 *            double with no fused multiply-add; its interpolation stencil
 *            must lie inside the h layers (layers floor(u_z) - 1 .. + 2 for
 *            tricubic, floor(u_z) .. + 1 for trilinear), else CMB3D_EINVAL.
 *   flags    CMB3D_FLAG_NO_SORT, ALLOW_WRAP (accepted; x and y always wrap),
 *            STAGE_TIMING, AUTOTUNE (y and x shapes), NO_PRUNE, PIPELINE;
 *            FUSED_YX and FP16_GEMM give CMB3D_EUNSUPPORTED.
 * The plan is used with the same calls as a 3-D plan: cmb3d_set_spectrum,
 * cmb3d_realize_sample(_to_host), cmb3d_realize_field (h x N x N floats),
 * cmb3d_draw_spectrum (the hybrid layers T^[z][m_y][m_x'], h x N x N/2
 * float2, m_x' = 0 packing T^(0, .) + i T^(N/2, .)), cmb3d_stage_times (the
 * draw of the correlated layers is reported as stage 0).  Batches of 2-D
 * plans run map by map.
 */
int cmb3d_plan_2d(cmb3d_plan_t* out, int N, int M, int h, double L, double r, double z0,
                  const double* pix_xyz, int64_t npix, int interp, uint32_t flags);

/*
 * The per-(m_x, m_y) factors of the 2-D method (host only): for every
 * q = m_x^2 + m_y^2 in [0, 2 (N/2)^2] reached by m_x in [0, N/2], m_y signed
 * in (-N/2, N/2], out[(q h + z) h + i] = S[z][i], the symmetric square root
 * (eigendecomposition, cyclic Jacobi in FP64, negative eigenvalues set to 0)
 * of Gamma_ij = sum_{m_z < M} P_box(m) cos(2 pi m_z (i - j) / M) with
 * P_box(m) = P_inf(|k|) (2 pi / dp)^3 / (M N^2), dp = L / N,
 * k = (2 pi m_x/(N dp), 2 pi m_y/(N dp), 2 pi m_z/(M dp)) (paper Eq. 2.11 for
 * an N x N x M box) and P_box(0) = 0; unreached q are zero.  P_inf is linear
 * in k between the n nodes (k, pk) as in cmb3d_set_spectrum.  out: host,
 * (2 (N/2)^2 + 1) h^2 floats.
 */
int cmb3d_gamma_sqrt_table(int N, int M, int h, double L, const double* k, const double* pk, int n, float* out);

/*
 * Set the box spectrum (paper Sec. II.A-C).
 *
 *   kind = CMB3D_SPEC_PK: x[0..n) are strictly increasing k >= 0 and y[0..n)
 *     the values P_inf(k) >= 0 (host pointers, copied).  P_inf is linear in k
 *     between nodes, equal to y[0] below x[0] and zero above x[n-1].
 *     nkbins and fit_err are ignored (fit_err, if not NULL, is set to 0).
 *   kind = CMB3D_SPEC_CL: x[0..n) are multipoles l >= 2 (integers, increasing)
 *     and y[0..n) the target C_l > 0.  P_inf >= 0 is fitted on nkbins uniform
 *     k nodes on [0, sqrt(3) pi N / L] by non-negative least squares on the
 *     relation C_l = 16 pi^2 int k^2 P(k) j_l(k r)^2 dk (relative residuals);
 *     nkbins must be in [8, 4096].  fit_err, if not NULL, receives the maximum
 *     relative error of the forward-projected C_l.
 * Then P_box(q) = P_inf(2 pi sqrt(q) / L) (2 pi / L)^3 (Eq. 2.11 with M = N)
 * is tabulated for q = 0 .. 3 (N/2)^2 and the table sqrt(P_box / 2) is
 * uploaded (one synchronous host-to-device copy).  On a plan of the 2-D
 * method (cmb3d_plan_2d) the uploaded table is instead the factor table of
 * cmb3d_gamma_sqrt_table for the plan's N, M, h and L ((2 (N/2)^2 + 1) h^2
 * floats, built on the host cores).
 * Errors: CMB3D_EINVAL for bad arrays, CMB3D_ENOMEM if the host table cannot
 * be allocated, CMB3D_ECUDA for the upload.
 */
int cmb3d_set_spectrum(cmb3d_plan_t plan, int kind, const double* x, const double* y,
                       int n, int nkbins, double* fit_err);

/*
 * Host-only form of the C_l inversion of cmb3d_set_spectrum(CMB3D_SPEC_CL),
 * needing no GPU: fits P_inf >= 0 on nk uniform nodes of [0, sqrt(3) pi N / L]
 * for a sphere of radius r.
 *   ell, cl     host arrays of n multipoles (integers >= 2, increasing) and
 *               C_l > 0.
 *   knodes_out  host array of nk doubles receiving the k nodes.
 *   pk_out      host array of nk doubles receiving P_inf at the nodes.
 *   fit_err     may be NULL; receives the maximum relative C_l error.
 * Errors: CMB3D_EINVAL for bad arguments; CMB3D_EUNSUPPORTED if the
 * non-negative least-squares iteration does not converge.
 */
int cmb3d_fit_pk(const double* ell, const double* cl, int n, int N, double L, double r, int nk,
                 double* knodes_out, double* pk_out, double* fit_err);

/*
 * The forward relation on a hat basis (host only): out[i * nk + j] =
 * 16 pi^2 int k^2 hat_j(k) j_l(k r)^2 dk for l = ell[i], so that for P_inf
 * linear between the nodes, C_l = sum_j out[i, j] P_inf(knodes[j]) (paper
 * Sec. II.A, Eq. 2.1 with Eq. 2.3-2.4 through the plane-wave expansion).
 * Gauss-Legendre (16 points per node interval), Miller's recurrence for j_l.
 *   ell     host, n integer multipoles >= 0; knodes host, nk increasing k >= 0;
 *   out     host, n * nk doubles (row-major).
 */
int cmb3d_cl_matrix(const double* ell, int n, const double* knodes, int nk, double r, double* out);

/*
 * The paper's linear-programming inversion (Sec. II.B), host only, needing no
 * GPU.  It finds P_inf >= 0 whose flat-space correlation function
 * xi_inf(r) = 4 pi int k P(k) sin(k r)/r dk (Eq. 2.4) matches the sphere's
 * xi_sph(theta) = sum_l (2l+1) C_l exp(-beam^2 l^2) P_l(cos theta) / (4 pi)
 * (Eq. 2.1 with the smoothing of Eq. 2.2) at the chords r = 2 R sin(theta/2)
 * (Eq. 2.3) of every separation in a polar cap of half-angle theta_max.
 *
 * Discretisation:
 *   - separations r_i = i dr, i < m = floor(r_max / dr) + 1, with r_max =
 *     2 R sin(theta_max) for theta_max <= pi/2 and 2 R beyond (the largest
 *     chord in the cap); targets b_i = xi_sph(theta_i), cos theta_i =
 *     1 - r_i^2 / (2 R^2);
 *   - unknowns x_j = P_inf(k_j) at k_j = j dk, j < nk = floor(kmax / dk);
 *     P_inf is linear between nodes and zero from k_nk = nk dk on, so the
 *     result is nk + 1 nodes whose last value is 0;
 *   - A_ij = 4 pi int k phi_j(k) sin(k r_i)/r_i dk (k^2 at r = 0), phi_j the
 *     hat function of node j, by Gauss-Legendre (16 points per interval).
 * The program (Eq. 2.5): minimise c^T x with c_j = sum_i A_ij subject to
 * A x >= b and x >= 0; its minimum is sum_i b_i exactly when A x = b has a
 * solution x >= 0.  Solved by a dense two-phase simplex on the dual problem
 * (n rows) in FP64.
 *
 *   ell, cl      host arrays of n multipoles (integers in [0, 100000],
 *                increasing) and C_l >= 0 (unsmoothed; beam is applied).
 *   R            sphere radius, > 0.
 *   theta_max    polar half-angle of the cap in radians, (0, pi].
 *   beam         Gaussian beam width b in radians (>= 0; 0 = no smoothing).
 *   dr, dk       separation and node steps; dr = 0 selects beam / 5 (then
 *                beam must be > 0) and dk = 0 selects 2 pi / (3 r_max), the
 *                paper's defaults.
 *   kmax         P_inf is zero above kmax (>= dk), e.g. sqrt(3) pi N / L, the
 *                largest |k| of a box.
 *
 * cmb3d_lp_system reports the program without solving it: m_out, nk_out
 * receive m and nk; each of r_out (m doubles), knodes_out (nk + 1), A_out
 * (m x nk, row-major) and b_out (m) may be NULL and is filled otherwise.
 *
 * cmb3d_fit_pk_lp solves it: knodes_out and pk_out (cap >= nk + 1 doubles
 * each) receive the nodes and P_inf at them, nk_out the count nk + 1;
 * objective (may be NULL) receives c^T x and xi_err (may be NULL)
 * max_i |(A x)_i - b_i| / |b_0|.  The result feeds
 * cmb3d_set_spectrum(CMB3D_SPEC_PK) unchanged.
 *
 * Errors: CMB3D_EINVAL for bad arguments or a too small cap;
 * CMB3D_EUNSUPPORTED above 1e6 separations, 1e5 nodes or 6.4e7 matrix or
 * tableau entries, or if the simplex reaches its pivot limit
 * (100 (m + nk) + 10000); CMB3D_ENOMEM if host memory runs out.
 */
int cmb3d_lp_system(const double* ell, const double* cl, int n, double R, double theta_max, double beam,
                    double dr, double dk, double kmax, int* m_out, int* nk_out, double* r_out,
                    double* knodes_out, double* A_out, double* b_out);
int cmb3d_fit_pk_lp(const double* ell, const double* cl, int n, double R, double theta_max, double beam,
                    double dr, double dk, double kmax, int cap, double* knodes_out, double* pk_out,
                    int* nk_out, double* objective, double* xi_err);

/*
 * Read back the plan's fitted P_inf(k) at n points (paper Sec. II.B output).
 *   k   host pointer, n abscissae (input); pk host pointer, n values (output).
 * Returns CMB3D_ENOSPEC before cmb3d_set_spectrum.
 */
int cmb3d_get_pk(cmb3d_plan_t plan, const double* k, double* pk, int n);

/*
 * One partial-sky map (paper Sec. II.D.1, the 3-D Fourier method): draw the
 * Gaussian Fourier coefficients of realization `seed`, inverse-FFT the box and
 * interpolate the field at the plan's pixels.
 *   out_dev  device pointer to npix floats, written in the caller's pixel
 *            order.  Caller-owned.
 *   stream   cudaStream_t the kernels are enqueued on (asynchronous).
 * Errors: CMB3D_ENOSPEC before cmb3d_set_spectrum; CMB3D_EINVAL for a NULL
 * out_dev with npix > 0; CMB3D_ECUDA if a launch fails.
 */
int cmb3d_realize_sample(cmb3d_plan_t plan, uint64_t seed, float* out_dev, void* stream);

/*
 * The same map delivered to host memory: enqueues cmb3d_realize_sample into the
 * plan's staging buffer, copies the npix floats to out_host (pinned memory is
 * fastest) and synchronises the stream before returning.  CMB3D_ETIMEOUT if a
 * bounded device-side wait gave up (tensor-core stage).
 */
int cmb3d_realize_sample_to_host(cmb3d_plan_t plan, uint64_t seed, float* out_host,
                                 void* stream);

/*
 * `count` maps delivered to host memory in one call, map i of realization
 * seeds[i] into outs_host[i] (npix floats each, the caller's pixel order).
 * The maps are computed in order on `stream` into two device staging buffers
 * used in turn; each map's download runs on a copy stream of the plan while
 * the kernels of the next map run, so with page-locked (pinned) host buffers
 * the copies overlap the computation.  Pageable host memory works but makes
 * each copy blocking.  Returns when every copy has completed (synchronises
 * `stream`).  The same host pointer may appear more than once; it then holds
 * the last of its maps.  The second staging buffer (4 npix bytes) and the
 * copy stream are created on the first call and kept by the plan.
 *   seeds      host array of count seeds; outs_host host array of count
 *              pointers.  count = 0 does nothing.
 * Errors: as cmb3d_realize_sample_to_host; CMB3D_EINVAL for NULL arrays or
 * a NULL output pointer with npix > 0.
 */
int cmb3d_realize_samples_to_host(cmb3d_plan_t plan, const uint64_t* seeds, int count, float* const* outs_host,
                                  void* stream);

/*
 * Many maps at once (batched form of Sec. II.D.1; the paper generates batches
 * of maps that reuse one set of precomputed quantities, Sec. II.D.2, Sec. IV).
 *   plans     host array of B distinct plans that share N, L, interp and
 *             device (their pixel sets and spectra may differ); each plan's
 *             box holds its realization.
 *   seeds     host array of B seeds; outs_dev host array of B device pointers,
 *             each to that plan's npix floats (caller's pixel order).
 * For N = 256 and 512 all B maps run in one persistent kernel launch, captured
 * once in a CUDA graph (kept in plans[0] for that plan set) and replayed: the
 * draw of one box overlaps with the FFT passes and gather of earlier ones.
 * With CMB3D_FLAG_AUTOTUNE on plans[0] the first call also times the
 * alternative form, a CUDA graph of two streams (draws on one, each box's
 * passes on a higher-priority one), and keeps the faster for this plan set and
 * these outputs.  Other N run the plans one after another.  Synchronises the stream before
 * returning.  Errors: CMB3D_EINVAL if the plans differ in N, L, interp or
 * device or repeat; CMB3D_ETIMEOUT if a bounded wait inside the persistent
 * kernel gave up (the context stays usable); CMB3D_ECUDA.  Batches that share
 * plans[0] must not run concurrently.
 */
int cmb3d_realize_sample_batch(const cmb3d_plan_t* plans, const uint64_t* seeds,
                               float* const* outs_dev, int B, void* stream);

/*
 * Test controls of the batched path (process-wide):
 *   spin_limit     polls of each bounded wait in the persistent kernel before
 *                  it gives up (0 restores the default, about 2 s);
 *   withhold_draw  != 0: draw items never report completion, so the waits that
 *                  depend on them must time out (fault injection);
 *   force_form     -1: the plan's choice; 0, 1: persistent kernel with two or
 *                  one resident blocks per SM; 2: the two-stream CUDA graph
 *                  (each box's draw on one stream, its y, x and gather passes
 *                  on a higher-priority stream).
 */
void cmb3d_batch_debug(uint32_t spin_limit, int withhold_draw, int force_form);

/*
 * Diagnostics of the intermediate stages of one realization (same seed
 * convention as cmb3d_realize_sample):
 *   cmb3d_draw_spectrum: the drawn half spectrum in the packed layout the
 *     kernels use, float2 [m_z][m_y][m_x'] with m_x' = 0 .. N/2-1, where entry
 *     m_x' = 0 holds T(0,m_y,m_z) + i T(N/2,m_y,m_z) and m_x' > 0 holds
 *     T(m_x',m_y,m_z).  spec_dev: device pointer to N*N*N/2 float2.
 *   cmb3d_realize_field: the real box field float[z][y][x] (N^3 floats).
 */
int cmb3d_draw_spectrum(cmb3d_plan_t plan, uint64_t seed, void* spec_dev, void* stream);
int cmb3d_realize_field(cmb3d_plan_t plan, uint64_t seed, float* field_dev, void* stream);

/*
 * Philox4x32-10 words exactly as the draw kernel computes them: for i < n,
 * out_dev[4i..4i+3] = Philox4x32-10(counter ctr_dev[4i..4i+3], key (seed lo,
 * seed hi)).  Device pointers; n >= 0.
 */
int cmb3d_philox4x32_10(const uint32_t* ctr_dev, uint64_t seed, uint32_t* out_dev,
                        int64_t n, void* stream);

/*
 * Per-stage device time in milliseconds accumulated since the last reset, for
 * plans made with CMB3D_FLAG_STAGE_TIMING (CMB3D_EINVAL otherwise).  ms[0..n)
 * receives stages CMB3D_STAGE_*; launches[0..n) (may be NULL) the number of
 * kernel launches timed per stage.  Synchronises on the recorded events.
 * reset != 0 clears the accumulators after reading.  Returns CMB3D_ETIMEOUT
 * (once) if a bounded device-side wait of the plan's kernels gave up since
 * the last check.
 */
int cmb3d_stage_times(cmb3d_plan_t plan, double* ms, int64_t* launches, int n, int reset);

/*
 * One partial-sky map with no device allocation, for callers that cannot call
 * cudaMalloc (code running inside another runtime that owns all device
 * memory, or behind an allocator that forbids new allocations).  The paper has
 * no counterpart to this call; it is the same computation as
 * cmb3d_realize_sample without a plan.
 *
 *   N        power of two, 8 <= N <= CMB3D_NOALLOC_MAX_N; larger N returns
 *            CMB3D_EUNSUPPORTED (the box does not fit the static scratch).
 *   L, r     box side and sphere radius, finite, > 0, L > 2r (CMB3D_EINVAL).
 *   pix_dev  device pointer, npix x 3 doubles (unit vectors, row-major).
 *            Not validated: a pixel whose grid coordinate is not finite (or
 *            beyond 4e15 cells) reads no memory and receives NaN.
 *   npix     0 <= npix < 2^31.
 *   interp   CMB3D_TRILINEAR or CMB3D_TRICUBIC.
 *   amp_dev  device pointer, 3 (N/2)^2 + 1 floats: amp[q] = sqrt(P_box(q) / 2)
 *            with P_box(q) = P_inf(2 pi sqrt(q) / L) (2 pi / L)^3, the table
 *            cmb3d_set_spectrum builds for a plan.
 *   out_dev  device pointer, npix floats, written in pixel order.
 * The box and twiddle tables live in one static __device__ array of about
 * 1 MiB.  The driver places it when it loads the library's module on a
 * device; under lazy module loading (CUDA_MODULE_LOADING=LAZY, the runtime's
 * default) that is the first call on that device, so a caller that must see
 * no allocation later makes one warm-up call at start-up.  The array stays
 * until the device's context is destroyed.  The first call in a device
 * context looks up the array's address and uploads the twiddle tables with a
 * synchronous copy, so make it before any stream capture; after
 * cudaDeviceReset the next call repeats that set-up.  Every call overwrites
 * the whole box before use, but all calls share the array: calls that overlap
 * on the GPU (other streams or threads) race and must be serialised by the
 * caller.  Calls no allocating routine of its own.  On a rejected call,
 * cmb3d_error_detail() gives the reason.
 */
#define CMB3D_NOALLOC_MAX_N 64
int cmb3d_realize_sample_noalloc(int N, double L, double r, const double* pix_dev, int64_t npix, int interp,
                                 const float* amp_dev, uint64_t seed, float* out_dev, void* stream);

/*
 * Test hooks (no counterpart in the paper):
 * cmb3d_debug_alloc_limit: from now on a plan (created or growing a second
 * box or staging buffer) whose device memory would pass `bytes` fails with
 * CMB3D_ENOMEM, as if cudaMalloc had run out, after freeing what it took; 0
 * removes the limit.  Process-wide, not thread-safe.
 * cmb3d_debug_poison_boxes: waits for the plan's work, then fills its box(es)
 * with the bit pattern 0xFFFFFFFF (NaN), so that a later map that read a box
 * entry no pass of its own had written would come out NaN.
 */
void cmb3d_debug_alloc_limit(int64_t bytes);
int cmb3d_debug_poison_boxes(cmb3d_plan_t plan);

/*
 * The kernel shapes the plan uses: sched[0] = draw+z variant, sched[1] = y
 * variant, sched[2] = x variant (both -1 when fused), sched[3] = fused y+x
 * variant (-1 when separate).  Variant 0 is each kernel's default shape; with
 * CMB3D_FLAG_AUTOTUNE the values are final after the first realization.
 * sched: host array of 4 ints.
 */
int cmb3d_plan_schedule(cmb3d_plan_t plan, int* sched);

/*
 * Pin the kernel shapes (same layout as cmb3d_plan_schedule; sched[3] >= 0
 * selects the fused y+x pass and then sched[1], sched[2] are ignored).  Turns
 * off a pending autotune.  CMB3D_EINVAL for a variant out of range or one the
 * plan's flags exclude.  sched: host array of 4 ints.
 */
int cmb3d_plan_set_schedule(cmb3d_plan_t plan, const int* sched);

/*
 * The batched form last built with `plan` as plans[0]: *form = -1 (none), 0
 * (persistent kernel; *variant = 0 two or 1 one resident blocks per SM) or 1
 * (two-stream CUDA graph).  form, variant: host pointers.
 */
int cmb3d_batch_schedule(cmb3d_plan_t plan, int* form, int* variant);

/* ------------------------------------------------------------------------
 * Learned inversion of the angular spectrum (stands in for the NNLS fit of
 * cmb3d_set_spectrum(CMB3D_SPEC_CL); the paper's inversion is the linear
 * program of Sec. II.B): an MLP maps log C_l to log P_inf at fixed k nodes.
 * Layers: `depth` hidden layers of `width` units with GELU (0.5 x (1 +
 * erf(x / sqrt 2))), then a linear output.  Inputs are normalised as
 * (log C_l - mu_l) / sd_l.  Training is label-free through the forward
 * relation A (n_in x n_out, the matrix of cmb3d_cl_matrix for the same l and
 * k nodes):  loss = mean over spectra and l of (log (A exp(y))_l - log C_l)^2.
 * GEMMs run on the tensor cores with BF16 operands and FP32 accumulation;
 * master weights, gradients and Adam moments are FP32.
 * Parameter layout (flat, FP32): for each layer W (out x in, row-major) then
 * its bias (out).
 * ------------------------------------------------------------------------ */
typedef struct cmb3d_mlp_s* cmb3d_mlp_t;

/*
 *   afwd       host, n_in x n_out doubles (forward relation, copied).
 *   mu, sd     host, n_in floats each, or NULL for 0 and 1.
 *   out_bias   host, n_out floats (initial output bias, e.g. log of a fitted
 *              P), or NULL for 0.  Weights start N(0, 1/fan_in) from `seed`.
 *   batch_cap  largest batch of train / loss_grad and the chunk of predict.
 */
int cmb3d_mlp_create(cmb3d_mlp_t* out, int n_in, int width, int depth, int n_out, const double* afwd,
                     const float* mu, const float* sd, const float* out_bias, int batch_cap, uint64_t seed);

/*
 * Adam (beta 0.9, 0.999, eps 1e-8, gradient clipped to global norm 1) over
 * `epochs` passes of shuffled batches of
 * `batch` rows of logcl_dev (device, n x n_in floats, log C_l); the epoch's
 * mean loss goes to epoch_loss_host[epoch] (may be NULL).  Synchronous.
 */
int cmb3d_mlp_train(cmb3d_mlp_t mlp, const float* logcl_dev, int64_t n, int epochs, int batch, float lr,
                    uint64_t seed, float* epoch_loss_host, void* stream);

/* log P_inf at the nodes for n spectra: logpk_dev (device, n x n_out floats). */
int cmb3d_mlp_predict(cmb3d_mlp_t mlp, const float* logcl_dev, int64_t n, float* logpk_dev, void* stream);

/*
 * Loss of n <= batch_cap spectra (host double) and, if grad_dev != NULL, the
 * gradient of the loss with respect to every parameter (device, flat layout).
 */
int cmb3d_mlp_loss_grad(cmb3d_mlp_t mlp, const float* logcl_dev, int64_t n, double* loss_host, float* grad_dev,
                        void* stream);

/*
 * Refine predicted spectra toward the non-negative least-squares optimum of
 * the forward relation (paper Sec. II.A: C_l = sum_j A[l, j] P(k_j)): P >= 0
 * minimising sum_l ((A P)_l / C_l - 1)^2, the objective of the NNLS inversion
 * of cmb3d_set_spectrum(CMB3D_SPEC_CL), by `iters` steps of accelerated
 * projected gradient (FISTA) started at exp(logpk), in the variable P / s with
 * s_j the inverse norm of column j of diag(1/C) A, step 1/L from a
 * `power_iters`-step power iteration (times 1.05).  Every product runs through
 * the network's BF16-operand, FP32-accumulate GEMM kernel.
 *   logcl_dev  device, n x n_in floats (log C_l);  logpk_dev  device, n x n_out (start, log P)
 *   pk_dev     device, n x n_out floats (result P, not log).  Synchronous.
 */
int cmb3d_mlp_refine(cmb3d_mlp_t mlp, const float* logcl_dev, const float* logpk_dev, int64_t n, int iters,
                     int power_iters, float* pk_dev, void* stream);

/* Parameter count (*count), read (get_host) and / or write (set_host), host floats. */
int cmb3d_mlp_params(cmb3d_mlp_t mlp, float* get_host, const float* set_host, int64_t* count);

void cmb3d_mlp_destroy(cmb3d_mlp_t mlp);

/*
 * Diagnostic: the network's matrix-product kernel on caller data, so that it
 * can be compared element by element with exact sums.  Every product of the
 * learned inversion runs through it (forward layers, the forward relation of
 * paper Sec. II.A, and the transposed products of the backward pass).
 *   out[m os0 + n os1] = f(alpha sum_k bf16(a[m as0 + k as1]) bf16(b[n bs0 + k bs1]) + bias[n])
 * for m < M, n < N, with operands rounded to bfloat16 (nearest, ties to even),
 * FP32 accumulation in tensor memory, f = GELU if gelu != 0 else identity,
 * bias (device, N floats) may be NULL.  a, b, out: device FP32, any strides
 * (so either operand may be transposed).  Synchronises on `stream`;
 * CMB3D_ETIMEOUT if a bounded wait for MMA completion gave up.
 */
int cmb3d_mlp_gemm(int M, int N, int K, const float* a, int64_t as0, int64_t as1, const float* b, int64_t bs0,
                   int64_t bs1, float alpha, const float* bias, int gelu, float* out, int64_t os0, int64_t os1,
                   void* stream);

/* Message of the most recent MLP error on the calling thread. */
const char* cmb3d_mlp_error_detail(void);

/* Plan properties: N, number of pixels, and device bytes owned by the plan. */
int cmb3d_plan_info(cmb3d_plan_t plan, int* N, int64_t* npix, int64_t* device_bytes);

/*
 * Extent of the pruned transform a sky map uses (the paper sizes its box to
 * the cap, Sec. II.C; here the cubic box is kept and only the part the
 * pixels' interpolation stencils read is transformed): *planes = z-planes the
 * y pass covers, *rows = (z, y) rows the x pass covers.  Without pruning
 * (CMB3D_FLAG_NO_PRUNE, N < 128, or stencils touching every row) N and N^2.
 * cmb3d_realize_field always transforms the whole box.  Host pointers; either
 * may be NULL.
 */
int cmb3d_plan_prune_info(cmb3d_plan_t plan, int64_t* planes, int64_t* rows);

/*
 * Reals the x pass of a sky map stores: for each row it covers, only the
 * column blocks (N/32 columns each) that the pixels' interpolation stencils
 * read are written back (the gather reads nothing else).  N^3 (N^2 h for the
 * 2-D method) without pruning.  *reals: host pointer.
 */
int cmb3d_plan_x_stored(cmb3d_plan_t plan, int64_t* reals);

/*
 * Host-only (no device, no allocation on any GPU): the extents of the pruned
 * transform (the part of the cubic box the cap's pixels read, the GPU form of
 * the cap-sized box of Sec. II.C) that a 3-D plan with the same arguments
 * would build from its pixels, counts[0..3] = z-planes the
 * y pass covers, (z, y) rows the x pass covers, reals the x pass stores, and
 * gather runs (pixels of one base cell, at most 8 per run; 0 with
 * CMB3D_FLAG_NO_SORT).  Without pruning (CMB3D_FLAG_NO_PRUNE, N < 128, or
 * stencils on every row) N, N^2 and N^3.  Arguments and their checks as for
 * cmb3d_plan; counts: host array of 4.
 */
int cmb3d_pixel_tables_host(int N, double L, double r, const double* pix_xyz, int64_t npix, int interp,
                            uint32_t flags, int64_t* counts);

/* Release the plan and all device memory it owns (NULL is ignored). */
void cmb3d_destroy(cmb3d_plan_t plan);

/* Name of a status code (static string). */
const char* cmb3d_strerror(int status);

/* Message of the most recent error on the calling thread (static per thread). */
const char* cmb3d_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* CMB3D_H */
