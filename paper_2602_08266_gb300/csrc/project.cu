// Scene preparation and projection (the rasterizer's first stage).
//
// Scene preparation, once per scene and target: opacity sigma = sigmoid(rho),
// object probabilities p = softmax(o) (Sec. III-A.1), the confidence c_g of
// Eq. 7 or its object-centric form of Eq. 12, per-axis scales, the
// normalised quaternion, and the two exponent thresholds that turn the
// alpha cut-off (1/255) and clamp (0.99) into comparisons on the splat
// exponent:  sigma e^p < alpha_min  <=>  p < log(alpha_min / sigma).
//
// Projection, per (view, Gaussian): camera-space centre, EWA 2D covariance
// with dilation, conic, 3-sigma radius, tile rectangle and depth key, the
// number of the rectangle's tiles that pass tile_hit (the entries the
// duplication will emit), and the view-dependent colour from the real
// spherical harmonics.
//
// The key path (everything that decides culling, the tile rectangle, the
// depth key and the per-pixel alpha decisions) uses only correctly rounded
// single-precision operations in one fixed order (explicit __f*_rn
// intrinsics, so no contraction into FMA), which makes it reproducible bit
// for bit by any IEEE implementation following the same order.
#include <math.h>

#include "nbv_internal.cuh"

namespace nbv {
namespace {

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fd(float a, float b) { return __fdiv_rn(a, b); }

__global__ void k_scene_prep(DevScene s, Consts c, int target) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= s.n) return;
  const int KC = c.KC;
  // per-axis scale, rounded once from a double exp
  float sc[3];
  for (int k = 0; k < 3; ++k) sc[k] = (float)exp((double)s.logs_raw[3 * g + k]);
  // normalised quaternion in correctly rounded single precision
  const float q0 = s.q_raw[4 * g], q1 = s.q_raw[4 * g + 1], q2 = s.q_raw[4 * g + 2],
              q3 = s.q_raw[4 * g + 3];
  const float n2 = fa(fa(fa(fm(q0, q0), fm(q1, q1)), fm(q2, q2)), fm(q3, q3));
  const float nr = __fsqrt_rn(n2);
  s.qn[g] = make_float4(fd(q0, nr), fd(q1, nr), fd(q2, nr), fd(q3, nr));
  // opacity and the two exponent thresholds
  const double sig = 1.0 / (1.0 + exp(-(double)s.rho_raw[g]));
  const float sig32 = (float)sig;
  const float pw_skip = (float)log((double)c.alpha_min / (double)sig32);
  const float pw_clamp = (float)log((double)c.alpha_max / (double)sig32);
  const float* m = s.mu_raw + 3 * g;
  s.mu_sig[g] = make_float4(m[0], m[1], m[2], sig32);
  s.scale_skip[g] = make_float4(sc[0], sc[1], sc[2], pw_skip);
  // p = softmax(o) in single precision (values only: every decision that
  // depends on the logits is the argmax, taken on the logits themselves,
  // lowest id on ties); the largest term is exp(0) = 1, so max_k p_k = 1 / z
  // and the confidence takes z summed in double
  const float* o = s.obj_raw + (size_t)g * KC;
  int am = 0;
  for (int k = 1; k < KC; ++k)
    if (o[k] > o[am]) am = k;
  const float mx = o[am];
  double z = 0.0;
  for (int k = 0; k < KC; ++k) z += (double)expf(o[k] - mx);
  const float zi = (float)(1.0 / z);
  float* p = s.p + (size_t)g * KC;
  for (int k = 0; k < KC; ++k) p[k] = expf(o[k] - mx) * zi;
  const double pmax = 1.0 / z;
  const double ptgt = (target >= 0 && target < KC) ? (double)expf(o[target] - mx) / z : 0.0;
  // Eq. 7, or Eq. 12 when a target object is given
  double cg;
  if (target < 0)
    cg = pow(pmax, -(double)c.alpha_obj) * pow(sig, -(double)c.alpha_opa);
  else
    cg = (am == target) ? pow(ptgt, -(double)c.alpha_obj) * pow(sig, -(double)c.alpha_opa) : 0.0;
  s.aux[g] = make_float4(pw_clamp, (float)cg, nr, __int_as_float(am));
}

// Real spherical harmonics (Condon-Shortley phase) of a unit direction,
// index l*l + l + m, written as polynomials in (x, y, z).
__device__ __forceinline__ void sh_eval(int deg, float x, float y, float z, float* Y) {
  constexpr double kPi = 3.14159265358979323846;
  const float c0 = (float)(0.5 / 1.7724538509055160273);            // 1/(2 sqrt(pi))
  Y[0] = c0;
  if (deg < 1) return;
  const float c1 = (float)0.48860251190291992159;                     // sqrt(3/(4 pi))
  Y[1] = -c1 * y; Y[2] = c1 * z; Y[3] = -c1 * x;
  if (deg < 2) return;
  const float c2a = (float)(0.5 * 3.8729833462074168852 / 1.7724538509055160273);   // sqrt(15/pi)/2
  const float c2b = (float)(0.25 * 2.2360679774997896964 / 1.7724538509055160273);  // sqrt(5/pi)/4
  const float c2c = (float)(0.25 * 3.8729833462074168852 / 1.7724538509055160273);  // sqrt(15/pi)/4
  Y[4] = c2a * x * y;
  Y[5] = -c2a * y * z;
  Y[6] = c2b * (2.0f * z * z - x * x - y * y);
  Y[7] = -c2a * x * z;
  Y[8] = c2c * (x * x - y * y);
  if (deg < 3) return;
  const float c3a = (float)(0.25 * 2.3601743597065740);   // sqrt(35/(2 pi))/4
  const float c3b = (float)(0.5 * 5.7812228852811080);    // sqrt(105/pi)/2
  const float c3c = (float)(0.25 * 1.8281831978578629);   // sqrt(21/(2 pi))/4
  const float c3d = (float)(0.25 * 1.4927053303604616);   // sqrt(7/pi)/4
  const float c3e = (float)(0.25 * 5.7812228852811080);   // sqrt(105/pi)/4
  Y[9] = -c3a * y * (3.0f * x * x - y * y);
  Y[10] = c3b * x * y * z;
  Y[11] = -c3c * y * (4.0f * z * z - x * x - y * y);
  Y[12] = c3d * z * (2.0f * z * z - 3.0f * x * x - 3.0f * y * y);
  Y[13] = -c3c * x * (4.0f * z * z - x * x - y * y);
  Y[14] = c3e * z * (x * x - y * y);
  Y[15] = -c3a * x * (x * x - 3.0f * y * y);
  (void)kPi;
}

// What project_one does besides computing a slot's records.
enum ProjMode {
  kProjAll = 0,      // multi-view: records of every slot (tiles counted by k_count_tiles)
  kProjCount = 1,    // one view: records, radius and the number of rectangle tiles that pass tile_hit
  kProjMark = 2      // multi-view, active slots: records, and their tiles marked in the view's tile mark
};
// (Every slot of the multi-view pass with a mark: k_project_target.)

// Tile marks of the multi-view pass with an active subset.
struct TileMark {
  uint8_t* mark;            // [global tiles]
  int4* bb;                 // [views] bounding box of marked tiles {min x, min y, max x, max y}
  uint32_t base;            // the view's first global tile
  int lo_x, lo_y, hi_x, hi_y;   // kProjMark: the box of the tiles this slot marked (hi_x < 0: none)
};

// The key path of Gaussian g in camera cam: culling, the conic, radius and
// tile rectangle in correctly rounded single precision and a fixed order.
// With a box (the view's box of marked tiles) a slot whose conservative
// radius bound cannot reach it is dropped after the projected centre.
// False: no rectangle (culled, degenerate, off the grid or dropped).
struct KeyPath {
  float mx, my, A, B, C, tz, r;
  int4 rect;                // {x0, x1, y0, y1}
};

__device__ __forceinline__ bool key_path(const Consts& c, const DevCam& cam, const float4& ms, const float4& ss,
                                         const float4& qq, const int4* box, KeyPath& kp) {
  const float* R = cam.R;
  // ---- key path: correctly rounded single precision, fixed order
  const float tx = fa(fa(fa(fm(R[0], ms.x), fm(R[1], ms.y)), fm(R[2], ms.z)), cam.t[0]);
  const float ty = fa(fa(fa(fm(R[3], ms.x), fm(R[4], ms.y)), fm(R[5], ms.z)), cam.t[1]);
  const float tz = fa(fa(fa(fm(R[6], ms.x), fm(R[7], ms.y)), fm(R[8], ms.z)), cam.t[2]);
  if (!(tz > c.near_z)) return false;
  const float xr = fd(tx, tz), yr = fd(ty, tz);
  const float mx = fa(fm(cam.fx, xr), cam.cx);
  const float my = fa(fm(cam.fy, yr), cam.cy);
  const float limx = fm(c.guard, fd(fm(0.5f, (float)cam.W), cam.fx));
  const float limy = fm(c.guard, fd(fm(0.5f, (float)cam.H), cam.fy));
  const float xz = fminf(limx, fmaxf(-limx, xr));
  const float yz = fminf(limy, fmaxf(-limy, yr));
  if (box != nullptr) {
    // Early rejection of a slot whose rectangle cannot reach the view's box
    // of marked tiles, before the rest of the key path. lambda_max of the 2D
    // covariance is at most its trace + sqrt(0.1) (the square root's floor),
    // and the trace at most ||J||_F^2 s_max^2 + 2 dilation, with
    // ||J||_F^2 = (fx^2 (1 + xz^2) + fy^2 (1 + yz^2)) / tz^2 for the clamped
    // xz, yz above and s_max the largest scale (the rotation is orthonormal).
    // The bound on the radius (3 sqrt(lambda) rounded up) carries a 1%
    // margin and 2 pixels for the rounding of this ordinary float estimate,
    // so only slots with no tile in the box are dropped.
    const int4 bx = *box;
    if (bx.z < bx.x || bx.w < bx.y) return false;        // no marked tile in this view
    const float smax = fmaxf(ss.x, fmaxf(ss.y, ss.z));
    const float iz = 1.0f / tz;
    const float jx = cam.fx * iz, jy = cam.fy * iz;
    const float tr = (jx * jx * (1.0f + xz * xz) + jy * jy * (1.0f + yz * yz)) * (smax * smax) + 2.0f * c.dilation;
    const float rb = 3.0f * sqrtf(tr + 0.5f) * 1.01f + 2.0f;
    const float twb = (float)cam.TW, thb = (float)cam.TH;
    if (mx + rb < (float)bx.x * twb || mx - rb >= (float)(bx.z + 1) * twb || my + rb < (float)bx.y * thb ||
        my - rb >= (float)(bx.w + 1) * thb)
      return false;
  }
  const float txp = fm(xz, tz), typ = fm(yz, tz);
  const float tz2 = fm(tz, tz);
  const float j00 = fd(cam.fx, tz), j02 = -fd(fm(cam.fx, txp), tz2);
  const float j11 = fd(cam.fy, tz), j12 = -fd(fm(cam.fy, typ), tz2);
  float T0[3], T1[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T0[i] = fa(fm(j00, R[i]), fm(j02, R[6 + i]));
    T1[i] = fa(fm(j11, R[3 + i]), fm(j12, R[6 + i]));
  }
  const float w = qq.x, x = qq.y, y = qq.z, z = qq.w;
  float Rq[9];
  Rq[0] = fs(1.0f, fm(2.0f, fa(fm(y, y), fm(z, z))));
  Rq[1] = fm(2.0f, fs(fm(x, y), fm(w, z)));
  Rq[2] = fm(2.0f, fa(fm(x, z), fm(w, y)));
  Rq[3] = fm(2.0f, fa(fm(x, y), fm(w, z)));
  Rq[4] = fs(1.0f, fm(2.0f, fa(fm(x, x), fm(z, z))));
  Rq[5] = fm(2.0f, fs(fm(y, z), fm(w, x)));
  Rq[6] = fm(2.0f, fs(fm(x, z), fm(w, y)));
  Rq[7] = fm(2.0f, fa(fm(y, z), fm(w, x)));
  Rq[8] = fs(1.0f, fm(2.0f, fa(fm(x, x), fm(y, y))));
  const float sc[3] = {ss.x, ss.y, ss.z};
  float V[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) V[3 * i + j] = fm(Rq[3 * i + j], sc[j]);
  float Sg[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Sg[3 * i + j] = fa(fa(fm(V[3 * i], V[3 * j]), fm(V[3 * i + 1], V[3 * j + 1])),
                         fm(V[3 * i + 2], V[3 * j + 2]));
  float U0[3], U1[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    U0[j] = fa(fa(fm(T0[0], Sg[j]), fm(T0[1], Sg[3 + j])), fm(T0[2], Sg[6 + j]));
    U1[j] = fa(fa(fm(T1[0], Sg[j]), fm(T1[1], Sg[3 + j])), fm(T1[2], Sg[6 + j]));
  }
  const float a = fa(fa(fa(fm(U0[0], T0[0]), fm(U0[1], T0[1])), fm(U0[2], T0[2])), c.dilation);
  const float b = fa(fa(fm(U0[0], T1[0]), fm(U0[1], T1[1])), fm(U0[2], T1[2]));
  const float cc = fa(fa(fa(fm(U1[0], T1[0]), fm(U1[1], T1[1])), fm(U1[2], T1[2])), c.dilation);
  const float det = fs(fm(a, cc), fm(b, b));
  if (!(det > 0.0f)) return false;
  const float A = fd(cc, det), B = fd(-b, det), C = fd(a, det);
  const float mid = fm(0.5f, fa(a, cc));
  const float lam = fa(mid, __fsqrt_rn(fmaxf(0.1f, fs(fm(mid, mid), det))));
  const float r = ceilf(fm(3.0f, __fsqrt_rn(lam)));
  const float twf = (float)cam.TW, thf = (float)cam.TH;
  const float fx0 = floorf(fd(fs(mx, r), twf)), fx1 = fa(floorf(fd(fa(mx, r), twf)), 1.0f);
  const float fy0 = floorf(fd(fs(my, r), thf)), fy1 = fa(floorf(fd(fa(my, r), thf)), 1.0f);
  const int x0 = (int)fminf(fmaxf(fx0, 0.0f), (float)cam.GX);
  const int x1 = (int)fminf(fmaxf(fx1, 0.0f), (float)cam.GX);
  const int y0 = (int)fminf(fmaxf(fy0, 0.0f), (float)cam.GY);
  const int y1 = (int)fminf(fmaxf(fy1, 0.0f), (float)cam.GY);
  if (x0 >= x1 || y0 >= y1) return false;
  kp.mx = mx; kp.my = my; kp.A = A; kp.B = B; kp.C = C; kp.tz = tz; kp.r = r;
  kp.rect = make_int4(x0, x1, y0, y1);
  return true;
}

// The records of a slot with entries: {mx, my, skip and clamp thresholds},
// {A, B, C, sigma}, the view-dependent colour (real SH, ordinary single
// precision) with camera z, the rectangle and the depth bits.
template <int DEG>
__device__ __forceinline__ void write_records(const DevScene& s, const DevCam& cam, int64_t g, const float4& ms,
                                              const float4& ss, const float4& ax, const KeyPath& kp,
                                              const DevProj& pr, size_t o) {
  const float mx = kp.mx, my = kp.my, A = kp.A, B = kp.B, C = kp.C, tz = kp.tz;
  const int x0 = kp.rect.x, x1 = kp.rect.y, y0 = kp.rect.z, y1 = kp.rect.w;
  // ---- view-dependent colour (values; ordinary single precision)
  float dv[3] = {ms.x - cam.campos[0], ms.y - cam.campos[1], ms.z - cam.campos[2]};
  const float il = rsqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
  // the degree is a template argument, so the basis stays in registers
  constexpr int NB = (DEG + 1) * (DEG + 1);
  float Y[16];
  sh_eval(DEG, dv[0] * il, dv[1] * il, dv[2] * il, Y);
  // SH coefficients as 16-byte vector loads: 3 nb floats per Gaussian start
  // 16-byte aligned when 3 nb is a multiple of 4 (SH degree 1 and 3)
  const float* shg = s.sh + (size_t)g * NB * 3;
  float rgb[3] = {0.5f, 0.5f, 0.5f};
  if constexpr ((NB * 3) % 4 == 0) {
    const float4* sh4 = reinterpret_cast<const float4*>(shg);
#pragma unroll
    for (int q = 0; q < (NB * 3) / 4; ++q) {
      const float4 v4 = __ldg(sh4 + q);
      const float e[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = 4 * q + u, k = idx / 3, ch = idx - 3 * k;
        rgb[ch] += Y[k] * e[u];
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < NB; ++k)
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) rgb[ch] += Y[k] * shg[3 * k + ch];
  }
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) rgb[ch] = fmaxf(rgb[ch], 0.0f);
  pr.r0[o] = make_float4(mx, my, ss.w, ax.x);
  pr.r1[o] = make_float4(A, B, C, ms.w);
  pr.r2[o] = make_float4(rgb[0], rgb[1], rgb[2], tz);
  pr.rect[o] = make_int4(x0, x1, y0, y1);
  pr.zbits[o] = __float_as_uint(tz);
}

// Project Gaussian g into camera cam; the records go to slot o of pr (see
// ProjMode for what else).
template <int kMode, int DEG>
__device__ __forceinline__ void project_one(const DevScene& s, const Consts& c, const DevCam& cam, int64_t g,
                                            const DevProj& pr, size_t o, TileMark* tm = nullptr) {
  const float4 ms = s.mu_sig[g];
  const float4 ss = s.scale_skip[g];
  const float4 qq = s.qn[g];
  const float4 ax = s.aux[g];
  if (kMode == kProjCount) {
    pr.touched[o] = 0u;
    pr.radius[o] = 0.0f;
  }
  pr.rect[o] = make_int4(-1, -1, -1, -1);
  pr.zbits[o] = 0u;
  KeyPath kp;
  if (!key_path(c, cam, ms, ss, qq, nullptr, kp)) return;
  const float mx = kp.mx, my = kp.my, A = kp.A, B = kp.B, C = kp.C;
  const int x0 = kp.rect.x, x1 = kp.rect.y, y0 = kp.rect.z, y1 = kp.rect.w;
  write_records<DEG>(s, cam, g, ms, ss, ax, kp, pr, o);
  if (kMode == kProjMark) {
    // mark this active splat's tiles and grow the view's box around them
    const float bc = -__fdiv_rn(B, C), ba = -__fdiv_rn(B, A);
    int lo_x = 0x7fffffff, lo_y = 0x7fffffff, hi_x = -1, hi_y = -1;
    for (int tyi = y0; tyi < y1; ++tyi)
      for (int txi = x0; txi < x1; ++txi)
        if (tile_hit(A, B, C, mx, my, ss.w, bc, ba, txi, tyi, cam.TW, cam.TH)) {
          uint8_t* mk = tm->mark + tm->base + (uint32_t)(tyi * cam.GX + txi);
          if (*mk == 0) *mk = 1;     // most tiles are marked by many splats: read before writing
          lo_x = min(lo_x, txi); hi_x = max(hi_x, txi);
          lo_y = min(lo_y, tyi); hi_y = max(hi_y, tyi);
        }
    tm->lo_x = lo_x; tm->lo_y = lo_y; tm->hi_x = hi_x; tm->hi_y = hi_y;   // the caller merges them into the box
  }
  if (kMode == kProjCount) {
    pr.radius[o] = kp.r;
    uint32_t hits = 0;
    const float bc = -__fdiv_rn(B, C), ba = -__fdiv_rn(B, A);
    for (int tyi = y0; tyi < y1; ++tyi)
      for (int txi = x0; txi < x1; ++txi)
        hits += tile_hit(A, B, C, mx, my, ss.w, bc, ba, txi, tyi, cam.TW, cam.TH) ? 1u : 0u;
    pr.touched[o] = hits;
  }
}

template <int DEG>
__global__ void k_project(DevScene s, Consts c, DevCam cam, DevProj pr) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= s.n) return;
  project_one<kProjCount, DEG>(s, c, cam, g, pr, (size_t)g);
}

// All views at once, one thread per (view, Gaussian): view blockIdx.y, slot
// v n + g; consecutive threads take consecutive Gaussians of one view, so
// every record load and store is coalesced and the camera is the block's.
template <int DEG, int kMode>
__global__ void __launch_bounds__(256) k_project_views(DevScene s, Consts c, const DevCam* __restrict__ cams,
                                                       DevProj pr) {
  __shared__ DevCam cam;
  const int v = blockIdx.y;
  if (threadIdx.x == 0) cam = cams[v];
  __syncthreads();
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= s.n) return;
  project_one<kMode, DEG>(s, c, cam, g, pr, (size_t)v * s.n + g);
}

// Every (view, Gaussian) slot of the multi-view pass with a target: the key
// path (dropping slots that cannot reach the view's box of marked tiles),
// the number of marked tiles inside the box that pass tile_hit (each thread
// walks its own rectangle: with the rectangles cut to the box, packing the
// warp's tiles into shared rounds measured slower), and the records of the
// slots with at least one.
template <int DEG>
__global__ void __launch_bounds__(256) k_project_target(DevScene s, Consts c, const DevCam* __restrict__ cams,
                                                        DevProj pr, const uint8_t* __restrict__ mark,
                                                        const int4* __restrict__ bb,
                                                        const uint32_t* __restrict__ tile_base) {
  __shared__ DevCam cam;
  const int v = blockIdx.y;
  if (threadIdx.x == 0) cam = cams[v];
  __syncthreads();
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= s.n) return;
  const size_t o = (size_t)v * s.n + g;
  pr.touched[o] = 0u;                            // records are read only for slots with entries
  const float4 ms = s.mu_sig[g];
  const float4 ss = s.scale_skip[g];
  const int4 box = bb[v];
  KeyPath kp;
  if (!key_path(c, cam, ms, ss, s.qn[g], &box, kp)) return;
  const int4 r = clip_rect(kp.rect, box);
  if (r.x < 0) return;
  const float bc = -__fdiv_rn(kp.B, kp.C), ba = -__fdiv_rn(kp.B, kp.A);
  const uint32_t base = tile_base[v];
  uint32_t hits = 0;
  for (int tyi = r.z; tyi < r.w; ++tyi)
    for (int txi = r.x; txi < r.y; ++txi)
      hits += (mark[base + (uint32_t)(tyi * cam.GX + txi)] != 0 &&
               tile_hit(kp.A, kp.B, kp.C, kp.mx, kp.my, ss.w, bc, ba, txi, tyi, cam.TW, cam.TH))
                  ? 1u
                  : 0u;
  if (hits == 0) return;
  pr.touched[o] = hits;
  write_records<DEG>(s, cam, g, ms, ss, s.aux[g], kp, pr, o);
}

// Active slots of the multi-view pass (thread per (view, active slot)):
// records, and their tiles marked with the view's box of marked tiles.
template <int DEG>
__global__ void __launch_bounds__(256) k_project_active(DevScene s, Consts c, const DevCam* __restrict__ cams,
                                                        int nv, DevProj pr, uint8_t* mark, int4* bb,
                                                        const uint32_t* __restrict__ tile_base) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= s.n_act * nv) return;
  const int v = (int)(i / s.n_act);
  const int64_t g = s.act[i - (int64_t)v * s.n_act];
  TileMark tm{mark, bb + v, tile_base[v], 0x7fffffff, 0x7fffffff, -1, -1};
  project_one<kProjMark, DEG>(s, c, cams[v], g, pr, (size_t)v * s.n + g, &tm);
  // merge into the view's box: one set of atomics per view present in the warp
  const unsigned peers = __match_any_sync(__activemask(), v);
  const int lo_x = __reduce_min_sync(peers, tm.lo_x), lo_y = __reduce_min_sync(peers, tm.lo_y);
  const int hi_x = __reduce_max_sync(peers, tm.hi_x), hi_y = __reduce_max_sync(peers, tm.hi_y);
  if ((threadIdx.x & 31) == __ffs(peers) - 1 && hi_x >= 0) {
    int* b = reinterpret_cast<int*>(bb + v);
    atomicMin(b, lo_x);
    atomicMin(b + 1, lo_y);
    atomicMax(b + 2, hi_x);
    atomicMax(b + 3, hi_y);
  }
}

}  // namespace

int launch_project_views(const DevScene& s, const Consts& c, const DevCam* cams, int nv, const DevProj& pr,
                         cudaStream_t st) {
  if (s.n <= 0 || nv <= 0) return 0;
  const int bs = 256;
  const dim3 grid((unsigned)((s.n + bs - 1) / bs), (unsigned)nv);
  switch (c.deg) {
    case 0: k_project_views<0, kProjAll><<<grid, bs, 0, st>>>(s, c, cams, pr); break;
    case 1: k_project_views<1, kProjAll><<<grid, bs, 0, st>>>(s, c, cams, pr); break;
    case 2: k_project_views<2, kProjAll><<<grid, bs, 0, st>>>(s, c, cams, pr); break;
    default: k_project_views<3, kProjAll><<<grid, bs, 0, st>>>(s, c, cams, pr); break;
  }
  return 1;
}

namespace {
__global__ void k_bbox_reset(int4* __restrict__ bb, int nv) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < nv) bb[v] = make_int4(0x7fffffff, 0x7fffffff, -1, -1);
}
}  // namespace

int launch_project_target(const DevScene& s, const Consts& c, const DevCam* cams, int nv, const DevProj& pr,
                          uint8_t* mark, int64_t ntiles, int4* bb, const uint32_t* tile_base, cudaStream_t st) {
  if (s.n <= 0 || nv <= 0) return 0;
  cudaMemsetAsync(mark, 0, (size_t)ntiles, st);
  k_bbox_reset<<<(nv + 255) / 256, 256, 0, st>>>(bb, nv);
  int l = 1;
  const int bs = 256;
  const int64_t na = s.n_act * nv;
  if (na > 0) {
    const unsigned ga = (unsigned)((na + bs - 1) / bs);
    switch (c.deg) {
      case 0: k_project_active<0><<<ga, bs, 0, st>>>(s, c, cams, nv, pr, mark, bb, tile_base); break;
      case 1: k_project_active<1><<<ga, bs, 0, st>>>(s, c, cams, nv, pr, mark, bb, tile_base); break;
      case 2: k_project_active<2><<<ga, bs, 0, st>>>(s, c, cams, nv, pr, mark, bb, tile_base); break;
      default: k_project_active<3><<<ga, bs, 0, st>>>(s, c, cams, nv, pr, mark, bb, tile_base); break;
    }
    ++l;
  }
  const dim3 grid((unsigned)((s.n + bs - 1) / bs), (unsigned)nv);
  switch (c.deg) {
    case 0: k_project_target<0><<<grid, bs, 0, st>>>(s, c, cams, pr, mark, bb, tile_base); break;
    case 1: k_project_target<1><<<grid, bs, 0, st>>>(s, c, cams, pr, mark, bb, tile_base); break;
    case 2: k_project_target<2><<<grid, bs, 0, st>>>(s, c, cams, pr, mark, bb, tile_base); break;
    default: k_project_target<3><<<grid, bs, 0, st>>>(s, c, cams, pr, mark, bb, tile_base); break;
  }
  return l + 1;
}

namespace {
// Input check of the n loaded Gaussians: bit 0 of *flag for a non-finite
// parameter, bit 1 for an all-zero quaternion (OR-ed over the grid).
__global__ void k_check_inputs(const float* __restrict__ mu, const float* __restrict__ logs,
                               const float* __restrict__ q, const float* __restrict__ rho,
                               const float* __restrict__ sh, const float* __restrict__ obj, int64_t n, int nsh,
                               int KC, int* __restrict__ flag) {
  int bits = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += stride) {
    bool ok = true;
    for (int i = 0; i < 3; ++i) ok = ok && isfinite(mu[3 * g + i]) && isfinite(logs[3 * g + i]);
    const float q0 = q[4 * g], q1 = q[4 * g + 1], q2 = q[4 * g + 2], q3 = q[4 * g + 3];
    ok = ok && isfinite(q0) && isfinite(q1) && isfinite(q2) && isfinite(q3) && isfinite(rho[g]);
    if (q0 == 0.0f && q1 == 0.0f && q2 == 0.0f && q3 == 0.0f) bits |= 2;
    for (int i = 0; i < nsh; ++i) ok = ok && isfinite(sh[g * nsh + i]);
    for (int i = 0; i < KC; ++i) ok = ok && isfinite(obj[g * KC + i]);
    if (!ok) bits |= 1;
  }
  bits = __reduce_or_sync(0xffffffffu, bits);
  if ((threadIdx.x & 31) == 0 && bits != 0) atomicOr(flag, bits);
}
}  // namespace

int launch_check_inputs(const float* mu, const float* logs, const float* q, const float* rho, const float* sh,
                        const float* obj, int64_t n, int nsh, int KC, int* flag, cudaStream_t st) {
  if (n <= 0) return 0;
  const int bs = 256;
  int64_t nb = (n + bs - 1) / bs;
  const int64_t cap = (int64_t)device_sm_count() * 16;
  if (nb > cap) nb = cap;
  k_check_inputs<<<(unsigned)nb, bs, 0, st>>>(mu, logs, q, rho, sh, obj, n, nsh, KC, flag);
  return 1;
}

namespace {
__global__ void k_active_flags(DevScene s, uint32_t* __restrict__ flags) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g < s.n) flags[g] = s.aux[g].y > 0.0f ? 1u : 0u;
}

__global__ void k_active_scatter(DevScene s, const uint32_t* __restrict__ flags, const uint32_t* __restrict__ off,
                                 int* __restrict__ slot, int* __restrict__ act) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= s.n) return;
  const bool on = flags[g] != 0u;
  slot[g] = on ? (int)off[g] : -1;
  if (on) act[off[g]] = (int)g;
}
}  // namespace

int launch_active_flags(const DevScene& s, uint32_t* flags, cudaStream_t st) {
  if (s.n <= 0) return 0;
  k_active_flags<<<(unsigned)((s.n + 255) / 256), 256, 0, st>>>(s, flags);
  return 1;
}

int launch_active_scatter(const DevScene& s, const uint32_t* flags, const uint32_t* offsets, int* slot, int* act,
                          cudaStream_t st) {
  if (s.n <= 0) return 0;
  k_active_scatter<<<(unsigned)((s.n + 255) / 256), 256, 0, st>>>(s, flags, offsets, slot, act);
  return 1;
}

int launch_scene_prep(const DevScene& s, const Consts& c, int target, cudaStream_t st) {
  if (s.n <= 0) return 0;
  const int bs = 128;
  k_scene_prep<<<(unsigned)((s.n + bs - 1) / bs), bs, 0, st>>>(s, c, target);
  return 1;
}

int launch_project(const DevScene& s, const Consts& c, const DevCam& cam, const DevProj& pr,
                   cudaStream_t st) {
  if (s.n <= 0) return 0;
  const int bs = 256;
  const unsigned grid = (unsigned)((s.n + bs - 1) / bs);
  switch (c.deg) {
    case 0: k_project<0><<<grid, bs, 0, st>>>(s, c, cam, pr); break;
    case 1: k_project<1><<<grid, bs, 0, st>>>(s, c, cam, pr); break;
    case 2: k_project<2><<<grid, bs, 0, st>>>(s, c, cam, pr); break;
    default: k_project<3><<<grid, bs, 0, st>>>(s, c, cam, pr); break;
  }
  return 1;
}

}  // namespace nbv
