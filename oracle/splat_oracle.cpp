// splat_oracle.cpp -- plain, slow CPU oracle of the differentiable tile-based
// RGB-D Gaussian rasterizer (MAC-Ego3D, arXiv 2412.09723).
//
// TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
// call this file: it is used by tests/, by __graft_entry__.smoke() and by the
// cpu_baseline / reference leg of bench.py.  It shares no code, header or
// constant table with the CUDA library; both sides are written separately from
// the same written specification of the operation order.
//
// What it computes (paper anchors):
//   * map representation: Gaussians with mean x, covariance Sigma (from a
//     scale vector and a rotation quaternion), opacity lambda and colour c
//     (Sec. 3.3, and Suppl. C.1 for the scale vector s_i);
//   * the rendering equation of Sec. 3.3: I(p) = sum_i c_i f_i(p)
//     prod_{j<i} (1 - f_j(p)), read as the product c_i * f_i(p), with f_i the
//     projected Gaussian's alpha at pixel p (the 3DGS definition the paper
//     cites);
//   * rendered depth D (Sec. 3.5 "Optimization", the depth term of the loss)
//     and the silhouette / final transmittance;
//   * the gradient of a per-pixel upstream gradient through all of it, to the
//     Gaussian parameters (mapping, Sec. 3.4 step 4) and to the SE(3) camera
//     pose (render-driven tracking / alignment, Sec. 3.5 steps 3-4);
//   * the L1 colour + depth loss of Eq. (optim) (L1 terms only);
//   * association of two renders by per-pixel maximum-weight Gaussian IDs
//     (Sec. 3.5 step 2, read as render-based pairing);
//   * Adam on resident parameters (the SplaTAM-style optimizer of Sec. 3.4).
//
// The paper is silent on every rasterizer constant; the readings used here
// (16x16 tiles, alpha cap 0.99, alpha floor 1/255, stop at T < 1e-4, +0.3
// low-pass, EWA clamp 1.3 tan(fov/2), near plane 0.2, pixel centres at +0.5,
// 3-sigma radius) are fixed in one written specification shared by name with
// the GPU path.
//
// Precision.  Every step is templated on the scalar type.  The float
// instantiation takes every discrete decision (culling, tile rectangle, sort
// order, alpha skip/stop, maximum-weight ID) in float with the specified
// operation order (-ffp-contract=off; std::fma exactly where the
// specification says fma), so that integer outputs can be compared
// bit-exactly.  Its exp is the project exp below (Cody & Waite range
// reduction + degree-7 Taylor polynomial).  The double instantiation uses
// std::exp and serves finite-difference checks of the adjoint.
//
// Pins (tests/test_oracle_*.py): project exp vs math.exp (ulp bound); single
// isotropic Gaussian closed form; hand-computed 2- and 3-Gaussian composites
// (tests/golden/); zero-opacity invariant; brute-force tile membership and
// depth order; central finite differences of the double adjoint for every
// parameter and the pose; L1 loss and Adam closed forms; brute-force
// association.  No function here is left unpinned.
//
// Threads.  The parity build is single-threaded (compiled without -fopenmp,
// every loop below runs in source order).  Built with -fopenmp, the same
// source is the timed CPU baseline: the projection runs over Gaussians and
// the per-tile sorts over tiles in parallel (same results), the forward
// render over tiles (same results), and the adjoint over tiles with one
// screen-space gradient buffer per thread, summed in thread order afterwards
// (the per-pixel arithmetic is unchanged; only the grouping of the sums over
// pixels and Gaussians differs).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>

#if defined(_OPENMP)
#include <omp.h>
#endif

namespace {

// ----------------------------------------------------------------------------
// Project exp (float).  Cody & Waite range reduction x = k ln2 + r with a
// two-part ln2, then exp(r) by a degree-7 Taylor polynomial in Horner form
// (coefficients 1/j!), then scaling by 2^k built from the exponent bits.
// Domain: x > 88 -> +inf, x < -87 -> 0, NaN -> NaN.
// ----------------------------------------------------------------------------
float exp_cw(float x) {
  if (x != x) return x;
  if (x > 88.0f) return std::numeric_limits<float>::infinity();
  if (x < -87.0f) return 0.0f;
  const float k = std::rint(x * 1.44269502f);
  float r = std::fma(-k, 0.693145751953125f, x);
  r = std::fma(-k, 1.42860677e-06f, r);
  float p = 1.98412701e-04f;           // 1/7!
  p = std::fma(p, r, 1.38888892e-03f); // 1/6!
  p = std::fma(p, r, 8.33333377e-03f); // 1/5!
  p = std::fma(p, r, 4.16666679e-02f); // 1/4!
  p = std::fma(p, r, 1.66666672e-01f); // 1/3!
  p = std::fma(p, r, 0.5f);            // 1/2!
  p = std::fma(p, r, 1.0f);
  p = std::fma(p, r, 1.0f);
  const int32_t ki = (int32_t)k;
  const uint32_t bits = (uint32_t)(ki + 127) << 23;
  float scale;
  std::memcpy(&scale, &bits, 4);
  return p * scale;
}

template <typename T> T act_exp(T x);
template <> float act_exp<float>(float x) { return exp_cw(x); }
template <> double act_exp<double>(double x) { return std::exp(x); }

template <typename T> inline T fma_(T a, T b, T c) { return std::fma(a, b, c); }

uint32_t float_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}

// Fixed constants of the specification (paper silent; 3DGS-style readings).
constexpr int TILE = 16;
template <typename T> struct K {
  static T alpha_cap() { return T(0.99); }
  static T alpha_min() { return T(1.0) / T(255.0); }
  static T tile_alpha() { return T(0.99) / T(255.0); }
  static T t_stop() { return T(1e-4); }
  static T lowpass() { return T(0.3); }
  static T clip() { return T(1.3); }
};
// In float the constants must be the float literals of the specification.
template <> struct K<float> {
  static float alpha_cap() { return 0.99f; }
  static float alpha_min() { return 1.0f / 255.0f; }
  static float tile_alpha() { return 0.99f / 255.0f; }
  static float t_stop() { return 1e-4f; }
  static float lowpass() { return 0.3f; }
  static float clip() { return 1.3f; }
};

template <typename T> struct Cam {
  int width, height;
  T fx, fy, cx, cy, znear;
  T maxdist;  // > 0: candidate selection by distance from the camera (Sec. 3.4 step 1)
  int tiles_x() const { return (width + TILE - 1) / TILE; }
  int tiles_y() const { return (height + TILE - 1) / TILE; }
};

// Per-Gaussian projection result (step O1).  radius == 0 means culled.
template <typename T> struct Proj {
  T u = 0, v = 0, z = 0, lam = 0;
  T cov_a = 0, cov_b = 0, cov_c = 0;  // 2D covariance incl. low-pass
  T con_a = 0, con_b = 0, con_c = 0;  // its inverse (the conic)
  T lam_max = 0;                      // larger eigenvalue of the 2D covariance
  T txz = 0, tyz = 0;                 // unclamped x/z, y/z
  int radius = 0;
  int rect[4] = {0, 0, 0, 0};  // xmin, ymin, xmax, ymax (tiles, half open)
  int tiles = 0;
};

// Intermediates of the activation + camera transform, recomputed for the adjoint.
template <typename T> struct Fwd3 {
  T s[3];      // scales
  T qn[4];     // normalised quaternion (w, x, y, z)
  T qnorm;     // |q| (0 => identity rotation)
  T R[3][3];   // rotation of the normalised quaternion
  T M[3][3];   // R diag(s)
  T Sig[3][3]; // 3D covariance M M^T
  T p[3];      // camera-space mean W x + t
  T J[2][3];   // EWA Jacobian
  T Tm[2][3];  // J W
  T tx, ty;    // clamped (x/z)*z, (y/z)*z
  bool clamp_x, clamp_y;
};

template <typename T>
void activation_camera(const T* x, const T* ls, const T* q, const T* w2c,
                       const Cam<T>& cam, Fwd3<T>& f) {
  // scales: s = exp(log_s)
  for (int k = 0; k < 3; ++k) f.s[k] = act_exp<T>(ls[k]);
  // quaternion normalisation (w, x, y, z); zero norm -> identity rotation
  const T n2 = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
  if (n2 == T(0)) {
    f.qnorm = T(0);
    f.qn[0] = T(1); f.qn[1] = T(0); f.qn[2] = T(0); f.qn[3] = T(0);
  } else {
    f.qnorm = std::sqrt(n2);
    for (int k = 0; k < 4; ++k) f.qn[k] = q[k] / f.qnorm;
  }
  const T r = f.qn[0], a = f.qn[1], b = f.qn[2], c = f.qn[3];
  const T one = T(1), two = T(2);
  f.R[0][0] = one - two * (b * b + c * c);
  f.R[0][1] = two * (a * b - r * c);
  f.R[0][2] = two * (a * c + r * b);
  f.R[1][0] = two * (a * b + r * c);
  f.R[1][1] = one - two * (a * a + c * c);
  f.R[1][2] = two * (b * c - r * a);
  f.R[2][0] = two * (a * c - r * b);
  f.R[2][1] = two * (b * c + r * a);
  f.R[2][2] = one - two * (a * a + b * b);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) f.M[i][j] = f.R[i][j] * f.s[j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      f.Sig[i][j] = (f.M[i][0] * f.M[j][0] + f.M[i][1] * f.M[j][1]) + f.M[i][2] * f.M[j][2];
  // camera transform p = W x + t  (w2c row-major 4x4)
  for (int i = 0; i < 3; ++i)
    f.p[i] = ((w2c[4 * i + 0] * x[0] + w2c[4 * i + 1] * x[1]) + w2c[4 * i + 2] * x[2]) + w2c[4 * i + 3];
  (void)cam;
}

// O1: activation, camera transform, EWA projection, radius and tile rect.
template <typename T>
Proj<T> project_one(const T* x, const T* ls, const T* q, T logit, const T* w2c,
                    const Cam<T>& cam, Fwd3<T>* keep = nullptr) {
  Proj<T> P;
  Fwd3<T> f;
  activation_camera(x, ls, q, w2c, cam, f);
  const T z = f.p[2];
  if (!(z > cam.znear)) {  // near-plane cull (also rejects NaN)
    if (keep) *keep = f;
    return P;
  }
  if (cam.maxdist > T(0)) {  // distance selection: |p|^2 = (p0 p0 + p1 p1) + p2 p2 against maxdist^2
    const T d2 = (f.p[0] * f.p[0] + f.p[1] * f.p[1]) + f.p[2] * f.p[2];
    if (d2 > cam.maxdist * cam.maxdist) {
      if (keep) *keep = f;
      return P;
    }
  }
  // EWA Jacobian with the guard-band clamp of x/z and y/z
  const T tan_x = T(cam.width) / (T(2) * cam.fx);
  const T tan_y = T(cam.height) / (T(2) * cam.fy);
  const T lim_x = K<T>::clip() * tan_x;
  const T lim_y = K<T>::clip() * tan_y;
  const T txz = f.p[0] / z;
  const T tyz = f.p[1] / z;
  const T txz_c = std::min(lim_x, std::max(-lim_x, txz));
  const T tyz_c = std::min(lim_y, std::max(-lim_y, tyz));
  f.clamp_x = !(txz >= -lim_x && txz <= lim_x);
  f.clamp_y = !(tyz >= -lim_y && tyz <= lim_y);
  f.tx = txz_c * z;
  f.ty = tyz_c * z;
  const T zz = z * z;
  f.J[0][0] = cam.fx / z;
  f.J[0][1] = T(0);
  f.J[0][2] = -(cam.fx * f.tx) / zz;
  f.J[1][0] = T(0);
  f.J[1][1] = cam.fy / z;
  f.J[1][2] = -(cam.fy * f.ty) / zz;
  // Tm = J W (row 0 uses J00, J02; row 1 uses J11, J12)
  for (int j = 0; j < 3; ++j) {
    f.Tm[0][j] = f.J[0][0] * w2c[0 * 4 + j] + f.J[0][2] * w2c[2 * 4 + j];
    f.Tm[1][j] = f.J[1][1] * w2c[1 * 4 + j] + f.J[1][2] * w2c[2 * 4 + j];
  }
  // Sigma2 = Tm Sigma Tm^T : first U = Tm Sigma, then U Tm^T
  T U[2][3];
  for (int a = 0; a < 2; ++a)
    for (int j = 0; j < 3; ++j)
      U[a][j] = (f.Tm[a][0] * f.Sig[0][j] + f.Tm[a][1] * f.Sig[1][j]) + f.Tm[a][2] * f.Sig[2][j];
  const T s00 = (U[0][0] * f.Tm[0][0] + U[0][1] * f.Tm[0][1]) + U[0][2] * f.Tm[0][2];
  const T s01 = (U[0][0] * f.Tm[1][0] + U[0][1] * f.Tm[1][1]) + U[0][2] * f.Tm[1][2];
  const T s11 = (U[1][0] * f.Tm[1][0] + U[1][1] * f.Tm[1][1]) + U[1][2] * f.Tm[1][2];
  const T ca = s00 + K<T>::lowpass();
  const T cb = s01;
  const T cc = s11 + K<T>::lowpass();
  const T det = ca * cc - cb * cb;
  if (keep) *keep = f;
  if (!(det > T(0))) return P;
  const T u = cam.fx * txz + cam.cx;
  const T v = cam.fy * tyz + cam.cy;
  const T mid = T(0.5) * (ca + cc);
  const T disc = mid * mid - det;
  const T lmax = mid + std::sqrt(std::max(disc, T(0)));
  const T rr = std::ceil(T(3) * std::sqrt(lmax));
  // O2: tile rectangle, half open, clamped to the tile grid
  const T tilef = T(TILE);
  const T gx = T(cam.tiles_x()), gy = T(cam.tiles_y());
  auto clampi = [](T val, T hi) { return (int)std::min(std::max(val, T(0)), hi); };
  const int xmin = clampi(std::floor((u - rr) / tilef), gx);
  const int ymin = clampi(std::floor((v - rr) / tilef), gy);
  // exclusive max: the tile of the last pixel centre <= u + r, plus one
  const int xmax = clampi(std::floor((u + rr) / tilef) + T(1), gx);
  const int ymax = clampi(std::floor((v + rr) / tilef) + T(1), gy);
  const int tiles = (xmax - xmin) * (ymax - ymin);
  if (tiles == 0) return P;
  P.u = u; P.v = v; P.z = z;
  P.lam = T(1) / (T(1) + act_exp<T>(-logit));
  P.cov_a = ca; P.cov_b = cb; P.cov_c = cc;
  P.con_a = cc / det;
  P.con_b = -cb / det;
  P.con_c = ca / det;
  P.lam_max = lmax;
  P.txz = txz; P.tyz = tyz;
  P.radius = (int)rr;
  P.rect[0] = xmin; P.rect[1] = ymin; P.rect[2] = xmax; P.rect[3] = ymax;
  P.tiles = tiles;
  return P;
}

template <typename T> struct Scene {
  int64_t n;
  const T *mean, *log_scale, *quat, *logit, *rgb;
};

template <typename T>
std::vector<Proj<T>> project_all(const Scene<T>& S, const T* w2c, const Cam<T>& cam) {
  std::vector<Proj<T>> P((size_t)S.n);
#if defined(_OPENMP)
#pragma omp parallel for schedule(static)
#endif
  for (int64_t g = 0; g < S.n; ++g)
    P[g] = project_one<T>(S.mean + 3 * g, S.log_scale + 3 * g, S.quat + 4 * g, S.logit[g], w2c, cam);
  return P;
}

// O2 + O3: per-tile candidate lists ordered by (depth, gid).  The depth order
// in float is the order of the float bit patterns (depth > 0).
// Only tile rows [ty0, ty1) are filled (all rows by default).
// Tile membership.  A tile of the Gaussian's rect can hold a contributor only
// if some point of its 16 x 16 rectangle of pixel centres reaches
// opacity * exp(-Q/2) >= 0.99/255, Q = a dx^2 + 2 b dx dy + c dy^2 (the conic
// of the projection): below 1/255 every pixel skips the Gaussian.  Q is convex,
// so its minimum over the rectangle is 0 with the centre inside, else on an
// edge, where it is a 1-D quadratic minimised in closed form.  The operation
// order is part of the specification (the decision must be the same in float
// on every implementation).
bool g_exact_tiles = true;  // test switch: false keeps whole rects

template <typename T>
bool tile_reaches(const Proj<T>& p, int tx, int ty) {
  const T xa = (T(TILE * tx) + T(0.5)) - p.u;
  const T xb = xa + T(15);
  const T ya = (T(TILE * ty) + T(0.5)) - p.v;
  const T yb = ya + T(15);
  if (xa <= T(0) && T(0) <= xb && ya <= T(0) && T(0) <= yb) return true;
  const T a = p.con_a, b = p.con_b, c = p.con_c;
  const T b2 = T(2) * b;
  const T ra = b / a, rc = b / c;
  T m = std::numeric_limits<T>::infinity();
  for (int e = 0; e < 2; ++e) {
    const T dy = e ? yb : ya;  // horizontal edge: minimiser dx = -(b/a) dy
    const T dx = std::fmin(xb, std::fmax(xa, -(ra * dy)));
    const T qh = ((a * dx) + (b2 * dy)) * dx + (c * dy) * dy;
    m = std::fmin(m, qh);
    const T ex = e ? xb : xa;  // vertical edge: minimiser dy = -(b/c) dx
    const T ey = std::fmin(yb, std::fmax(ya, -(rc * ex)));
    const T qv = (a * ex) * ex + ((b2 * ex) + (c * ey)) * ey;
    m = std::fmin(m, qv);
  }
  return p.lam * act_exp<T>(T(-0.5) * m) >= K<T>::tile_alpha();
}

// The member tiles of row ty: from the first to the last tile of the rect row
// that passes tile_reaches (the set of tiles meeting the ellipse within a
// band is contiguous; holes from rounding are filled by definition).  Returns
// false for an empty row.
template <typename T>
bool row_members(const Proj<T>& p, int ty, int& x0, int& x1) {
  if (!g_exact_tiles) {
    x0 = p.rect[0];
    x1 = p.rect[2] - 1;
    return x0 <= x1;
  }
  x0 = p.rect[0];
  while (x0 < p.rect[2] && !tile_reaches(p, x0, ty)) ++x0;
  if (x0 >= p.rect[2]) return false;
  x1 = p.rect[2] - 1;
  while (x1 > x0 && !tile_reaches(p, x1, ty)) --x1;
  return true;
}

template <typename T>
std::vector<std::vector<int32_t>> bin_all(const std::vector<Proj<T>>& P, const Cam<T>& cam, int ty0 = 0,
                                          int ty1 = 1 << 30) {
  const int ntx = cam.tiles_x(), nty = cam.tiles_y();
  std::vector<std::vector<int32_t>> bins((size_t)ntx * nty);
  for (size_t g = 0; g < P.size(); ++g) {
    const Proj<T>& p = P[g];
    if (p.tiles == 0) continue;
    for (int ty = std::max(p.rect[1], ty0); ty < std::min(p.rect[3], ty1); ++ty) {
      int x0, x1;
      if (!row_members(p, ty, x0, x1)) continue;
      for (int tx = x0; tx <= x1; ++tx) bins[(size_t)ty * ntx + tx].push_back((int32_t)g);
    }
  }
#if defined(_OPENMP)
#pragma omp parallel for schedule(dynamic, 8)
#endif
  for (int64_t t = 0; t < (int64_t)bins.size(); ++t)
    std::sort(bins[t].begin(), bins[t].end(), [&](int32_t i, int32_t j) {
      if (P[i].z != P[j].z) return P[i].z < P[j].z;
      return i < j;
    });
  return bins;
}

// One contributor of a pixel, recorded for the adjoint.
template <typename T> struct Contrib {
  int32_t g;
  T alpha, Tbefore, G, dx, dy;
  bool capped;
};

template <typename T> struct PixOut {
  T rgb[3], depth, sil, tfin;
  int ncontrib, maxid;
};

// FNV-1a over the discrete decisions (for the finite-difference checks).
struct Sig {
  uint64_t h = 1469598103934665603ull;
  void add(int64_t v) {
    for (int k = 0; k < 8; ++k) {
      h ^= (uint64_t)((v >> (8 * k)) & 0xff);
      h *= 1099511628211ull;
    }
  }
};

// O4: front-to-back compositing of one pixel over its tile's ordered list.
template <typename T>
PixOut<T> composite_pixel(int x, int y, const std::vector<int32_t>& list,
                          const std::vector<Proj<T>>& P, const T* rgb, const T* bg,
                          std::vector<Contrib<T>>* rec, Sig* sig) {
  const T px = T(x) + T(0.5);
  const T py = T(y) + T(0.5);
  T Tr = T(1);
  T C[3] = {T(0), T(0), T(0)};
  T D = T(0), Sl = T(0), wmax = T(0);
  int id = -1, last = 0;
  for (size_t j = 0; j < list.size(); ++j) {
    const int32_t g = list[j];
    const Proj<T>& p = P[g];
    const T dx = p.u - px;
    const T dy = p.v - py;
    // power = -0.5 a dx^2 - b dx dy - 0.5 c dy^2 in the specified order
    const T A = T(-0.5) * p.con_a;
    const T B = -p.con_b;
    const T Cc = T(-0.5) * p.con_c;
    const T power = fma_(Cc * dy, dy, dx * fma_(A, dx, B * dy));
    if (power > T(0)) continue;
    const T G = act_exp<T>(power);
    const T raw = p.lam * G;
    const T alpha = std::min(K<T>::alpha_cap(), raw);
    if (alpha < K<T>::alpha_min()) continue;
    const T test_T = Tr * (T(1) - alpha);
    if (test_T < K<T>::t_stop()) break;
    const T w = alpha * Tr;
    for (int k = 0; k < 3; ++k) C[k] = fma_(rgb[3 * g + k], w, C[k]);
    D = fma_(p.z, w, D);
    Sl = Sl + w;
    if (w > wmax) { wmax = w; id = g; }
    if (rec) rec->push_back(Contrib<T>{g, alpha, Tr, G, dx, dy, raw > K<T>::alpha_cap()});
    if (sig) sig->add((int64_t)j);
    Tr = test_T;
    last = (int)j + 1;
  }
  PixOut<T> o;
  for (int k = 0; k < 3; ++k) o.rgb[k] = fma_(Tr, bg[k], C[k]);
  o.depth = D;
  o.sil = Sl;
  o.tfin = Tr;
  o.ncontrib = last;
  o.maxid = id;
  if (sig) sig->add(-1 - (int64_t)last);
  return o;
}

template <typename T>
Cam<T> make_cam(const int32_t* ci, const T* cf) {
  Cam<T> c;
  c.width = ci[0]; c.height = ci[1];
  c.fx = cf[0]; c.fy = cf[1]; c.cx = cf[2]; c.cy = cf[3]; c.znear = cf[4]; c.maxdist = cf[5];
  return c;
}

template <typename T>
Scene<T> make_scene(int64_t n, const T* mean, const T* ls, const T* q, const T* logit, const T* rgb) {
  Scene<T> s;
  s.n = n; s.mean = mean; s.log_scale = ls; s.quat = q; s.logit = logit; s.rgb = rgb;
  return s;
}

// ---------------------------------------------------------------------------
// Forward render of one view.
// ---------------------------------------------------------------------------
// Pixel rows [row0, row1) are rendered (a band of the image; the rest of the
// outputs is left untouched).
template <typename T>
int render_fwd(const Scene<T>& S, const T* w2c, const Cam<T>& cam, const T* bg,
               T* out_rgb, T* out_depth, T* out_sil, T* out_tfin, int32_t* out_n,
               int32_t* out_id, uint64_t* signature, int64_t* n_pairs, int row0, int row1) {
  auto P = project_all(S, w2c, cam);
  auto bins = bin_all(P, cam, row0 / TILE, (row1 + TILE - 1) / TILE);
  const int ntx = cam.tiles_x();
  Sig sig;
  int64_t pairs = 0;
  for (size_t g = 0; g < P.size(); ++g) {
    sig.add(P[g].radius);
    for (int k = 0; k < 4; ++k) sig.add(P[g].rect[k]);
  }
  auto pixel = [&](int x, int y, Sig* sg) -> int64_t {
    const auto& list = bins[(size_t)(y / TILE) * ntx + (x / TILE)];
    PixOut<T> o = composite_pixel<T>(x, y, list, P, S.rgb, bg, nullptr, sg);
    const size_t i = (size_t)y * cam.width + x;
    for (int k = 0; k < 3; ++k) out_rgb[3 * i + k] = o.rgb[k];
    out_depth[i] = o.depth;
    out_sil[i] = o.sil;
    out_tfin[i] = o.tfin;
    out_n[i] = o.ncontrib;
    out_id[i] = o.maxid;
    return o.ncontrib;
  };
#if defined(_OPENMP)
  if (!signature) {  // timing build: tiles in parallel (every pixel computed as below)
    const int ty0 = row0 / TILE, ty1 = (row1 + TILE - 1) / TILE;
    const int64_t nt = (int64_t)(ty1 - ty0) * ntx;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : pairs)
    for (int64_t t = 0; t < nt; ++t) {
      const int ty = ty0 + (int)(t / ntx), tx = (int)(t % ntx);
      for (int y = std::max(row0, ty * TILE); y < std::min(row1, ty * TILE + TILE); ++y)
        for (int x = tx * TILE; x < std::min(cam.width, tx * TILE + TILE); ++x) pairs += pixel(x, y, nullptr);
    }
    if (n_pairs) *n_pairs = pairs;
    return 0;
  }
#endif
  for (int y = row0; y < row1; ++y)
    for (int x = 0; x < cam.width; ++x) pairs += pixel(x, y, signature ? &sig : nullptr);
  if (signature) *signature = sig.h;
  if (n_pairs) *n_pairs = pairs;
  return 0;
}

// ---------------------------------------------------------------------------
// O6: adjoint.  Per pixel: record the contributors front to back, then form
// dL/dalpha_i from suffix sums S_X = sum_{j>i} X_j w_j:
//   d(sum_j X_j w_j)/d alpha_i = X_i T_i - S_X / (1 - alpha_i),
//   d T_final / d alpha_i      = -T_final / (1 - alpha_i).
// Then per Gaussian the chain through alpha = min(cap, lam exp(power)),
// power(u, v, conic), the conic inverse, Sigma2 = (J W) Sigma (J W)^T + 0.3 I,
// the EWA Jacobian J(p) with its clamp, p = W x + t, Sigma = R S S^T R^T,
// the quaternion normalisation, s = exp(log_s) and lam = sigmoid(logit).
// The pose gradient is the 6-vector (rho, phi) of the left perturbation
// w2c <- exp(delta^) w2c:  dp = rho + phi x p,  dW = [phi]x W.
// ---------------------------------------------------------------------------
template <typename T> struct Grad2D {
  T du = 0, dv = 0, dca = 0, dcb = 0, dcc = 0, dlam = 0, dz = 0, drgb[3] = {0, 0, 0};
};

template <typename T>
void pixel_adjoint(const std::vector<Contrib<T>>& cs, const PixOut<T>& o, const T* gC, T gD,
                   T gS, const std::vector<Proj<T>>& P, const T* rgb, const T* bg,
                   std::vector<Grad2D<T>>& G2) {
  const size_t n = cs.size();
  // suffix sums S_X[i] = sum_{j > i} X_j w_j
  std::vector<T> SC0(n + 1, T(0)), SC1(n + 1, T(0)), SC2(n + 1, T(0)), SD(n + 1, T(0)), SS(n + 1, T(0));
  for (size_t ii = n; ii-- > 0;) {
    const Contrib<T>& c = cs[ii];
    const T w = c.alpha * c.Tbefore;
    SC0[ii] = SC0[ii + 1] + rgb[3 * c.g + 0] * w;
    SC1[ii] = SC1[ii + 1] + rgb[3 * c.g + 1] * w;
    SC2[ii] = SC2[ii + 1] + rgb[3 * c.g + 2] * w;
    SD[ii] = SD[ii + 1] + P[c.g].z * w;
    SS[ii] = SS[ii + 1] + w;
  }
  const T gbg = (gC[0] * bg[0] + gC[1] * bg[1]) + gC[2] * bg[2];
  for (size_t i = 0; i < n; ++i) {
    const Contrib<T>& c = cs[i];
    const Proj<T>& p = P[c.g];
    Grad2D<T>& d = G2[c.g];
    const T Ti = c.Tbefore;
    const T w = c.alpha * Ti;
    const T om = T(1) - c.alpha;
    const T* col = rgb + 3 * c.g;
    for (int k = 0; k < 3; ++k) d.drgb[k] += gC[k] * w;
    d.dz += gD * w;
    T dA = gC[0] * (col[0] * Ti - SC0[i + 1] / om) + gC[1] * (col[1] * Ti - SC1[i + 1] / om) +
           gC[2] * (col[2] * Ti - SC2[i + 1] / om);
    dA += gD * (p.z * Ti - SD[i + 1] / om);
    dA += gS * (Ti - SS[i + 1] / om);
    dA -= gbg * o.tfin / om;
    if (c.capped) continue;  // alpha = cap: no gradient to lam or power
    d.dlam += c.G * dA;
    const T dpow = p.lam * c.G * dA;
    d.du += dpow * (-(p.con_a * c.dx + p.con_b * c.dy));
    d.dv += dpow * (-(p.con_b * c.dx + p.con_c * c.dy));
    d.dca += dpow * (T(-0.5) * c.dx * c.dx);
    d.dcb += dpow * (-c.dx * c.dy);
    d.dcc += dpow * (T(-0.5) * c.dy * c.dy);
  }
}

template <typename T>
void project_adjoint(int64_t g, const Scene<T>& S, const T* w2c, const Cam<T>& cam,
                     const Grad2D<T>& d, T* d_mean, T* d_ls, T* d_q, T* d_logit, T* d_pose) {
  Fwd3<T> f;
  const Proj<T> p = project_one<T>(S.mean + 3 * g, S.log_scale + 3 * g, S.quat + 4 * g, S.logit[g], w2c, cam, &f);
  if (p.tiles == 0) return;
  const T z = f.p[2];
  // opacity
  d_logit[g] += d.dlam * p.lam * (T(1) - p.lam);
  // conic -> 2D covariance: gS2 = -Q gQ Q  (full symmetric matrices)
  const T Q[2][2] = {{p.con_a, p.con_b}, {p.con_b, p.con_c}};
  const T gQ[2][2] = {{d.dca, T(0.5) * d.dcb}, {T(0.5) * d.dcb, d.dcc}};
  T tmp[2][2], gS2[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) tmp[i][j] = Q[i][0] * gQ[0][j] + Q[i][1] * gQ[1][j];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) gS2[i][j] = -(tmp[i][0] * Q[0][j] + tmp[i][1] * Q[1][j]);
  // Sigma2 = Tm Sig Tm^T:  gTm = 2 gS2 Tm Sig ;  gSig = Tm^T gS2 Tm
  T TS[2][3];
  for (int a = 0; a < 2; ++a)
    for (int j = 0; j < 3; ++j) TS[a][j] = f.Tm[a][0] * f.Sig[0][j] + f.Tm[a][1] * f.Sig[1][j] + f.Tm[a][2] * f.Sig[2][j];
  T gTm[2][3];
  for (int a = 0; a < 2; ++a)
    for (int j = 0; j < 3; ++j) gTm[a][j] = T(2) * (gS2[a][0] * TS[0][j] + gS2[a][1] * TS[1][j]);
  T gSig[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T acc = T(0);
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) acc += f.Tm[a][i] * gS2[a][b] * f.Tm[b][j];
      gSig[i][j] = acc;
    }
  // Tm = J W:  gJ = gTm W^T ; gW (from Tm) = J^T gTm
  T W[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) W[i][j] = w2c[4 * i + j];
  T gJ[2][3];
  for (int a = 0; a < 2; ++a)
    for (int k = 0; k < 3; ++k) gJ[a][k] = gTm[a][0] * W[k][0] + gTm[a][1] * W[k][1] + gTm[a][2] * W[k][2];
  T gW[3][3];
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 3; ++j) gW[k][j] = f.J[0][k] * gTm[0][j] + f.J[1][k] * gTm[1][j];
  // J(z, tx, ty): J00 = fx/z, J02 = -fx tx/z^2, J11 = fy/z, J12 = -fy ty/z^2
  T gp[3] = {T(0), T(0), T(0)};
  const T z2 = z * z, z3 = z2 * z;
  T gz = -cam.fx / z2 * gJ[0][0] + T(2) * cam.fx * f.tx / z3 * gJ[0][2] - cam.fy / z2 * gJ[1][1] +
         T(2) * cam.fy * f.ty / z3 * gJ[1][2];
  const T gtx = -cam.fx / z2 * gJ[0][2];
  const T gty = -cam.fy / z2 * gJ[1][2];
  // tx = clamp(px/z) z : unclamped -> tx = px ; clamped -> tx = +-lim z
  if (!f.clamp_x) gp[0] += gtx; else gz += gtx * (f.tx / z);
  if (!f.clamp_y) gp[1] += gty; else gz += gty * (f.ty / z);
  // u = fx px/z + cx ; v = fy py/z + cy ; depth = z
  gp[0] += d.du * cam.fx / z;
  gz += -d.du * cam.fx * f.p[0] / z2;
  gp[1] += d.dv * cam.fy / z;
  gz += -d.dv * cam.fy * f.p[1] / z2;
  gz += d.dz;
  gp[2] += gz;
  // mean: p = W x + t
  for (int j = 0; j < 3; ++j) d_mean[3 * g + j] += W[0][j] * gp[0] + W[1][j] * gp[1] + W[2][j] * gp[2];
  // Sigma = M M^T: gM = 2 gSig M ; M = R diag(s)
  T gM[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) gM[i][j] = T(2) * (gSig[i][0] * f.M[0][j] + gSig[i][1] * f.M[1][j] + gSig[i][2] * f.M[2][j]);
  T gR[3][3];
  for (int j = 0; j < 3; ++j) {
    T gs = T(0);
    for (int i = 0; i < 3; ++i) {
      gs += gM[i][j] * f.R[i][j];
      gR[i][j] = gM[i][j] * f.s[j];
    }
    d_ls[3 * g + j] += gs * f.s[j];
  }
  // rotation of the normalised quaternion (r, a, b, c)
  if (f.qnorm > T(0)) {
    const T r = f.qn[0], a = f.qn[1], b = f.qn[2], c = f.qn[3];
    T gqn[4];
    gqn[0] = T(2) * (-c * gR[0][1] + b * gR[0][2] + c * gR[1][0] - a * gR[1][2] - b * gR[2][0] + a * gR[2][1]);
    gqn[1] = T(2) * (b * gR[0][1] + c * gR[0][2] + b * gR[1][0] - r * gR[1][2] + c * gR[2][0] + r * gR[2][1]) -
             T(4) * a * (gR[1][1] + gR[2][2]);
    gqn[2] = T(2) * (a * gR[0][1] + r * gR[0][2] + a * gR[1][0] + c * gR[1][2] - r * gR[2][0] + c * gR[2][1]) -
             T(4) * b * (gR[0][0] + gR[2][2]);
    gqn[3] = T(2) * (-r * gR[0][1] + a * gR[0][2] + r * gR[1][0] + b * gR[1][2] + a * gR[2][0] + b * gR[2][1]) -
             T(4) * c * (gR[0][0] + gR[1][1]);
    const T dot = f.qn[0] * gqn[0] + f.qn[1] * gqn[1] + f.qn[2] * gqn[2] + f.qn[3] * gqn[3];
    for (int k = 0; k < 4; ++k) d_q[4 * g + k] += (gqn[k] - f.qn[k] * dot) / f.qnorm;
  }
  // pose (left perturbation): rho += gp ; phi += p x gp + vee(gW W^T)
  if (d_pose) {
    T A[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) A[i][j] = gW[i][0] * W[j][0] + gW[i][1] * W[j][1] + gW[i][2] * W[j][2];
    d_pose[0] += gp[0];
    d_pose[1] += gp[1];
    d_pose[2] += gp[2];
    d_pose[3] += f.p[1] * gp[2] - f.p[2] * gp[1] + (A[2][1] - A[1][2]);
    d_pose[4] += f.p[2] * gp[0] - f.p[0] * gp[2] + (A[0][2] - A[2][0]);
    d_pose[5] += f.p[0] * gp[1] - f.p[1] * gp[0] + (A[1][0] - A[0][1]);
  }
}

template <typename T>
int render_bwd(const Scene<T>& S, const T* w2c, const Cam<T>& cam, const T* bg, const T* g_rgb,
               const T* g_depth, const T* g_sil, T* d_mean, T* d_ls, T* d_q, T* d_logit, T* d_rgb,
               T* d_pose, T* d2d, int row0, int row1) {
  auto P = project_all(S, w2c, cam);
  auto bins = bin_all(P, cam, row0 / TILE, (row1 + TILE - 1) / TILE);
  const int ntx = cam.tiles_x();
  std::vector<Grad2D<T>> G2((size_t)S.n);
  auto pixel = [&](int x, int y, std::vector<Contrib<T>>& rec, std::vector<Grad2D<T>>& G) {
    const auto& list = bins[(size_t)(y / TILE) * ntx + (x / TILE)];
    rec.clear();
    PixOut<T> o = composite_pixel<T>(x, y, list, P, S.rgb, bg, &rec, nullptr);
    const size_t i = (size_t)y * cam.width + x;
    const T gC[3] = {g_rgb[3 * i], g_rgb[3 * i + 1], g_rgb[3 * i + 2]};
    pixel_adjoint<T>(rec, o, gC, g_depth ? g_depth[i] : T(0), g_sil ? g_sil[i] : T(0), P, S.rgb, bg, G);
  };
#if defined(_OPENMP)
  // timing build: tiles in parallel, one screen-space gradient buffer per
  // thread, the buffers summed in thread order; then the projection adjoint
  // over Gaussians in parallel with one pose gradient per thread
  const int nth = omp_get_max_threads();
  std::vector<std::vector<Grad2D<T>>> G2t((size_t)nth);
  std::vector<T> pose_t((size_t)nth * 6, T(0));
  {
    const int ty0 = row0 / TILE, ty1 = (row1 + TILE - 1) / TILE;
    const int64_t nt = (int64_t)(ty1 - ty0) * ntx;
#pragma omp parallel
    {
      const int th = omp_get_thread_num();
      G2t[th].assign((size_t)S.n, Grad2D<T>());
      std::vector<Contrib<T>> rec;
#pragma omp for schedule(dynamic, 4)
      for (int64_t t = 0; t < nt; ++t) {
        const int ty = ty0 + (int)(t / ntx), tx = (int)(t % ntx);
        for (int y = std::max(row0, ty * TILE); y < std::min(row1, ty * TILE + TILE); ++y)
          for (int x = tx * TILE; x < std::min(cam.width, tx * TILE + TILE); ++x) pixel(x, y, rec, G2t[th]);
      }
#pragma omp for schedule(static)
      for (int64_t g = 0; g < S.n; ++g) {
        Grad2D<T>& d = G2[g];
        for (int k = 0; k < nth; ++k) {
          const Grad2D<T>& e = G2t[k][g];
          d.du += e.du; d.dv += e.dv; d.dca += e.dca; d.dcb += e.dcb; d.dcc += e.dcc;
          d.dlam += e.dlam; d.dz += e.dz;
          for (int c = 0; c < 3; ++c) d.drgb[c] += e.drgb[c];
        }
      }
#pragma omp for schedule(static)
      for (int64_t g = 0; g < S.n; ++g) {
        const Grad2D<T>& d = G2[g];
        for (int k = 0; k < 3; ++k) d_rgb[3 * g + k] += d.drgb[k];
        if (d2d) {
          T* o = d2d + 10 * g;
          o[0] = d.du; o[1] = d.dv; o[2] = d.dca; o[3] = d.dcb; o[4] = d.dcc;
          o[5] = d.dlam; o[6] = d.drgb[0]; o[7] = d.drgb[1]; o[8] = d.drgb[2]; o[9] = d.dz;
        }
        project_adjoint<T>(g, S, w2c, cam, d, d_mean, d_ls, d_q, d_logit, &pose_t[6 * (size_t)th]);
      }
    }
  }
  for (int k = 0; k < nth; ++k)
    for (int j = 0; j < 6; ++j) d_pose[j] += pose_t[6 * (size_t)k + j];
  return 0;
#endif
  std::vector<Contrib<T>> rec;
  for (int y = row0; y < row1; ++y)
    for (int x = 0; x < cam.width; ++x) pixel(x, y, rec, G2);
  for (int64_t g = 0; g < S.n; ++g) {
    const Grad2D<T>& d = G2[g];
    for (int k = 0; k < 3; ++k) d_rgb[3 * g + k] += d.drgb[k];
    if (d2d) {
      T* o = d2d + 10 * g;
      o[0] = d.du; o[1] = d.dv; o[2] = d.dca; o[3] = d.dcb; o[4] = d.dcc;
      o[5] = d.dlam; o[6] = d.drgb[0]; o[7] = d.drgb[1]; o[8] = d.drgb[2]; o[9] = d.dz;
    }
    project_adjoint<T>(g, S, w2c, cam, d, d_mean, d_ls, d_q, d_logit, d_pose);
  }
  return 0;
}

}  // namespace

// ============================================================================
// C ABI (host pointers; caller owns every buffer).
// Test switch: 0 keeps whole rects as tile members (the images must not change).
extern "C" void oracle_set_exact_tiles(int on) { g_exact_tiles = on != 0; }

// Threads the loops above use: 1 in the parity build; in the -fopenmp build
// the OpenMP maximum (OMP_NUM_THREADS, else every core), or `n` once set.
extern "C" int oracle_threads(void) {
#if defined(_OPENMP)
  return omp_get_max_threads();
#else
  return 1;
#endif
}
extern "C" void oracle_set_threads(int n) {
#if defined(_OPENMP)
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

// cam_i = {width, height}; cam_f = {fx, fy, cx, cy, z_near, max_dist}; w2c = 4x4 row-major.
// ============================================================================
extern "C" {

void oracle_exp_f32(int64_t n, const float* x, float* y) {
  for (int64_t i = 0; i < n; ++i) y[i] = exp_cw(x[i]);
}

#define ORACLE_PROJECT(SUF, T)                                                                   \
  int oracle_project_##SUF(int64_t n, const T* mean, const T* log_scale, const T* quat,          \
                           const T* logit, const T* w2c, const int32_t* cam_i, const T* cam_f,   \
                           T* xyzo, T* conic, T* cov, int32_t* radius, int32_t* rect,            \
                           int32_t* tiles) {                                                     \
    const Cam<T> cam = make_cam<T>(cam_i, cam_f);                                                \
    for (int64_t g = 0; g < n; ++g) {                                                            \
      const Proj<T> p = project_one<T>(mean + 3 * g, log_scale + 3 * g, quat + 4 * g, logit[g], \
                                       w2c, cam);                                                \
      xyzo[4 * g + 0] = p.u; xyzo[4 * g + 1] = p.v; xyzo[4 * g + 2] = p.z;                      \
      xyzo[4 * g + 3] = p.lam;                                                                   \
      conic[4 * g + 0] = p.con_a; conic[4 * g + 1] = p.con_b; conic[4 * g + 2] = p.con_c;        \
      conic[4 * g + 3] = T(0);                                                                   \
      if (cov) { cov[3 * g] = p.cov_a; cov[3 * g + 1] = p.cov_b; cov[3 * g + 2] = p.cov_c; }     \
      radius[g] = p.radius;                                                                      \
      for (int k = 0; k < 4; ++k) rect[4 * g + k] = p.rect[k];                                   \
      tiles[g] = p.tiles;                                                                        \
    }                                                                                            \
    return 0;                                                                                    \
  }
ORACLE_PROJECT(f32, float)
ORACLE_PROJECT(f64, double)

// Binning (O2 + O3) in float.  keys = (tile << 32) | float_bits(depth), vals = gid,
// flattened over tiles in tile order; ranges[2 t], ranges[2 t + 1] = [start, end)
// ((0, 0) for an empty tile).  Returns K; writes at most `capacity` entries.
int64_t oracle_bin_f32(int64_t n, const float* mean, const float* log_scale, const float* quat,
                       const float* logit, const float* w2c, const int32_t* cam_i,
                       const float* cam_f, int64_t capacity, uint64_t* keys, uint32_t* vals,
                       uint32_t* ranges) {
  const Cam<float> cam = make_cam<float>(cam_i, cam_f);
  Scene<float> S = make_scene<float>(n, mean, log_scale, quat, logit, nullptr);
  auto P = project_all(S, w2c, cam);
  auto bins = bin_all(P, cam);
  int64_t k = 0;
  for (size_t t = 0; t < bins.size(); ++t) {
    const int64_t start = k;
    for (int32_t g : bins[t]) {
      if (k < capacity) {
        keys[k] = ((uint64_t)t << 32) | (uint64_t)float_bits(P[g].z);
        vals[k] = (uint32_t)g;
      }
      ++k;
    }
    ranges[2 * t] = bins[t].empty() ? 0u : (uint32_t)start;
    ranges[2 * t + 1] = bins[t].empty() ? 0u : (uint32_t)k;
  }
  return k;
}

#define ORACLE_FWD(SUF, T)                                                                       \
  int oracle_render_fwd_##SUF(int64_t n, const T* mean, const T* log_scale, const T* quat,       \
                              const T* logit, const T* rgb, const T* w2c, const int32_t* cam_i,  \
                              const T* cam_f, const T* bg, T* out_rgb, T* out_depth, T* out_sil, \
                              T* out_tfin, int32_t* out_n, int32_t* out_id, uint64_t* signature, \
                              int64_t* n_pairs, int32_t row0, int32_t row1) {                    \
    const Cam<T> cam = make_cam<T>(cam_i, cam_f);                                                \
    Scene<T> S = make_scene<T>(n, mean, log_scale, quat, logit, rgb);                            \
    row0 = std::max(0, row0);                                                                    \
    row1 = std::min(cam.height, row1);                                                           \
    return render_fwd<T>(S, w2c, cam, bg, out_rgb, out_depth, out_sil, out_tfin, out_n, out_id,  \
                         signature, n_pairs, row0, row1);                                        \
  }
ORACLE_FWD(f32, float)
ORACLE_FWD(f64, double)

// Rows [row0, row1) of the image are rendered / differentiated (pass 0 and the height for
// the whole frame).
// Gradients are accumulated (+=) into caller-zeroed buffers.  d2d (optional) receives the
// per-Gaussian screen-space gradients [n,10] = du, dv, dconic_a, dconic_b, dconic_c,
// dlambda, drgb[3], ddepth.
#define ORACLE_BWD(SUF, T)                                                                        \
  int oracle_render_bwd_##SUF(int64_t n, const T* mean, const T* log_scale, const T* quat,        \
                              const T* logit, const T* rgb, const T* w2c, const int32_t* cam_i,   \
                              const T* cam_f, const T* bg, const T* g_rgb, const T* g_depth,      \
                              const T* g_sil, T* d_mean, T* d_log_scale, T* d_quat, T* d_logit,   \
                              T* d_rgb, T* d_pose, T* d2d, int32_t row0, int32_t row1) {          \
    const Cam<T> cam = make_cam<T>(cam_i, cam_f);                                                 \
    Scene<T> S = make_scene<T>(n, mean, log_scale, quat, logit, rgb);                             \
    row0 = std::max(0, row0);                                                                     \
    row1 = std::min(cam.height, row1);                                                            \
    return render_bwd<T>(S, w2c, cam, bg, g_rgb, g_depth, g_sil, d_mean, d_log_scale, d_quat,     \
                         d_logit, d_rgb, d_pose, d2d, row0, row1);                                \
  }
ORACLE_BWD(f32, float)
ORACLE_BWD(f64, double)

// L1 loss of Eq. (optim), L1 terms: L = w_rgb mean|C - C*| + w_depth mean|D - D*|,
// sign(0) = 0.  Writes dL/dC, dL/dD; returns L (summed in double).
double oracle_loss_l1_f32(int64_t npix, const float* rgb, const float* depth, const float* t_rgb,
                          const float* t_depth, float w_rgb, float w_depth, float* g_rgb,
                          float* g_depth) {
  double acc_c = 0.0, acc_d = 0.0;
  const float sc = w_rgb / (float)(3 * npix);
  const float sd = w_depth / (float)npix;
  for (int64_t i = 0; i < 3 * npix; ++i) {
    const float e = rgb[i] - t_rgb[i];
    acc_c += std::fabs((double)e);
    g_rgb[i] = e > 0.0f ? sc : (e < 0.0f ? -sc : 0.0f);
  }
  for (int64_t i = 0; i < npix; ++i) {
    const float e = depth[i] - t_depth[i];
    acc_d += std::fabs((double)e);
    g_depth[i] = e > 0.0f ? sd : (e < 0.0f ? -sd : 0.0f);
  }
  return (double)w_rgb * acc_c / (double)(3 * npix) + (double)w_depth * acc_d / (double)npix;
}

// Adam (textbook; bias-corrected), step = t >= 1.
void oracle_adam_f32(int64_t n, float* param, const float* grad, float* m, float* v, int32_t step,
                     float lr, float beta1, float beta2, float eps) {
  const float bc1 = 1.0f - std::pow(beta1, (float)step);
  const float bc2 = 1.0f - std::pow(beta2, (float)step);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0f - beta1) * grad[i];
    v[i] = beta2 * v[i] + (1.0f - beta2) * grad[i] * grad[i];
    const float mh = m[i] / bc1;
    const float vh = v[i] / bc2;
    param[i] = param[i] - lr * mh / (std::sqrt(vh) + eps);
  }
}

// Render-based association: the pixels where both renders have a maximum-weight
// Gaussian and both final transmittances are <= t_max give pairs (id_a, id_b);
// returned sorted by (id_a, id_b), unique, with the number of pixels per pair.
// Returns M; writes at most `capacity` pairs.
int64_t oracle_assoc(int64_t npix, const int32_t* id_a, const float* t_a, const int32_t* id_b,
                     const float* t_b, float t_max, int64_t capacity, int32_t* pairs,
                     int32_t* counts) {
  std::vector<uint64_t> v;
  for (int64_t i = 0; i < npix; ++i)
    if (id_a[i] >= 0 && id_b[i] >= 0 && t_a[i] <= t_max && t_b[i] <= t_max)
      v.push_back(((uint64_t)(uint32_t)id_a[i] << 32) | (uint64_t)(uint32_t)id_b[i]);
  std::sort(v.begin(), v.end());
  int64_t m = 0;
  for (size_t i = 0; i < v.size();) {
    size_t j = i;
    while (j < v.size() && v[j] == v[i]) ++j;
    if (m < capacity) {
      pairs[2 * m] = (int32_t)(v[i] >> 32);
      pairs[2 * m + 1] = (int32_t)(v[i] & 0xffffffffu);
      counts[m] = (int32_t)(j - i);
    }
    ++m;
    i = j;
  }
  return m;
}

}  // extern "C"
