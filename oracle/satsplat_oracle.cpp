/*
 * FP64 CPU oracle of the affine 2D-Gaussian-splat (surfel) rasterizer of SatSplat.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code, header
 * or constant with the CUDA path, and the CUDA path never calls it.
 *
 * It is the plain per-pixel definition, with no tiling and no sorting beyond
 * the visibility order the paper prescribes:
 *   - affine camera x = F [p; 1], split into B_xy, b_xy and the fixed depth row
 *     B_z = [0, 0, -1], b_z = max_altitude            (Sec. 3.1 Eq. affine_camera;
 *                                                      Sec. 3.2 Eq. decompose_affine_camera,
 *                                                      Eq. depth_affine_camera)
 *   - learnable delta F'_xy = F_xy + dF_xy            (Sec. 3.3)
 *   - sun camera B_sun = B'_xy (I - [0 0 s]), scaled to the shadow-map size
 *                                                      (Sec. 3.3 Eq. sun_camera_Bxy; Supp. A)
 *   - splat P(u,v) = p + s_u t_u u + s_v t_v v with [t_u t_v n] = R(q)
 *                                                      (Sec. 3.1 Eq. 2dgs_splat_param)
 *   - screen -> uv: u = Q x + q, Q = (B_xy R S')^-1, q = -Q (B_xy p + b_xy)
 *                                                      (Sec. 3.2 Eq. affine2dgs_screen2uv,
 *                                                      Eq. affine2dgs_Qq)
 *   - lower-bounded Gaussian G^ = max(G(u), G((x - c)/sigma)); when |det| is
 *     below the threshold only the screen-space term exists  (Sec. 3.2, degenerate solutions)
 *   - normal = last column of R, alpha-blended           (Sec. 3.2, normal definition)
 *   - front-to-back blending f = sum f_i a_i G^_i prod_{j<i} (1 - a_j G^_j) over
 *     splats ordered by the height-based depth of their centres   (Sec. 3.2 Eq. rasterization)
 *   - corrected albedo C A + c                           (Sec. 3.1 Eq. image_formation)
 *   - distortion of the blending weights along the ray: the sum over composited
 *     pairs j before i of 2 w_i w_j (z_i - z_j), w_i = a_i G^_i T_i and z_i the
 *     depth of the ray-splat intersection (the point-sample distortion loss that
 *     Supp. B adds to the training loss, in compositing order; it equals
 *     sum_{i,j} w_i w_j |z_i - z_j| when that order is the order of z)
 * Readings where the paper is silent (alpha threshold 1/255, clamp 0.99, early
 * stop at T < 1e-4 excluding the stopping splat, ties by splat index, pixel
 * centres at +0.5, depth at the intersection point, normal flipped to face the
 * sensor) are listed in the design notes; every constant comes in as an argument.
 *
 * The forward pass is templated on the scalar type so that a dual-number run
 * gives exact directional derivatives; the reverse-mode adjoint is written out
 * by hand in double and checked against it.
 */
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- camera record (doubles)
enum {
  C_F = 0, C_DF = 8, C_MAXALT = 16, C_W = 17, C_H = 18, C_COLOR = 19,
  C_PHI = 31, C_THETA = 32, C_SW = 33, C_SH = 34, C_SSCALE = 35, C_NUM = 36
};
// ---------------------------------------------------------------- options (doubles)
enum { O_SIGMA = 0, O_DETEPS = 1, O_AMIN = 2, O_AMAX = 3, O_TMIN = 4, O_NUM = 5 };

// ---------------------------------------------------------------- dual numbers
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double a) : v(a), d(0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual operator/(Dual a, Dual b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual exp(Dual a) { double e = std::exp(a.v); return {e, e * a.d}; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return {s, a.d / (2 * s)}; }
inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
using std::exp;
using std::sqrt;

template <class S> inline S lift(double v, const double* dir, int64_t i);
template <> inline double lift<double>(double v, const double*, int64_t) { return v; }
template <> inline Dual lift<Dual>(double v, const double* dir, int64_t i) {
  return Dual(v, dir ? dir[i] : 0.0);
}

// ---------------------------------------------------------------- scene
struct Scene {
  int64_t n;
  const double *means, *scales, *quats, *opac, *rgb;  // planar [C][n]
};
struct Dirs {  // tangent directions for the dual-number run (nullable)
  const double *means, *scales, *quats, *opac, *rgb, *dF, *color;
};

// ---------------------------------------------------------------- camera assembly (a1)
template <class S> struct Cam {
  S B[2][3], b[2];  // screen rows
  double maxalt;    // b_z
  double vs[3];     // unit viewing direction toward the sensor (z > 0)
  int W, H;
  bool sun;
  double S_, s[3];  // sun: resolution scale and flattening direction
};

template <class S>
Cam<S> assemble(const double* cam, const double* dF_dir, bool sun) {
  Cam<S> C;
  S Bp[2][3], bp[2];
  for (int i = 0; i < 2; ++i) {
    for (int j = 0; j < 3; ++j)
      Bp[i][j] = S(cam[C_F + 4 * i + j]) + lift<S>(cam[C_DF + 4 * i + j], dF_dir, 4 * i + j);
    bp[i] = S(cam[C_F + 4 * i + 3]) + lift<S>(cam[C_DF + 4 * i + 3], dF_dir, 4 * i + 3);
  }
  C.maxalt = cam[C_MAXALT];
  C.sun = sun;
  // viewing direction of the main camera: null space of B'_xy, B_x x B_y (Sec. 3.3)
  double d[3] = {val(Bp[0][1]) * val(Bp[1][2]) - val(Bp[0][2]) * val(Bp[1][1]),
                 val(Bp[0][2]) * val(Bp[1][0]) - val(Bp[0][0]) * val(Bp[1][2]),
                 val(Bp[0][0]) * val(Bp[1][1]) - val(Bp[0][1]) * val(Bp[1][0])};
  double dn = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  double sg = d[2] < 0 ? -1.0 : 1.0;
  for (int i = 0; i < 3; ++i) C.vs[i] = sg * d[i] / dn;
  if (!sun) {
    for (int i = 0; i < 2; ++i) {
      for (int j = 0; j < 3; ++j) C.B[i][j] = Bp[i][j];
      C.b[i] = bp[i];
    }
    C.W = (int)cam[C_W];
    C.H = (int)cam[C_H];
    C.S_ = 1.0;
    C.s[0] = C.s[1] = 0.0;
    C.s[2] = 0.0;
  } else {
    // s = (cos(phi)/tan(theta), sin(phi)/tan(theta), 1); B_sun = S * B' (I - s e3^T)   (Supp. A)
    double phi = cam[C_PHI], th = cam[C_THETA];
    double s[3] = {std::cos(phi) / std::tan(th), std::sin(phi) / std::tan(th), 1.0};
    double Sc = cam[C_SSCALE];
    for (int i = 0; i < 2; ++i) {
      for (int j = 0; j < 3; ++j) {
        S acc = S(0.0);
        for (int k = 0; k < 3; ++k) {
          double P = (k == j ? 1.0 : 0.0) - (j == 2 ? s[k] : 0.0);
          acc += Bp[i][k] * S(P);
        }
        C.B[i][j] = S(Sc) * acc;
      }
      C.b[i] = S(Sc) * bp[i];
    }
    C.W = (int)cam[C_SW];
    C.H = (int)cam[C_SH];
    C.S_ = Sc;
    for (int k = 0; k < 3; ++k) C.s[k] = s[k];
  }
  return C;
}

// ---------------------------------------------------------------- projection (a2)
template <class S> struct Proj {
  S o, rgb[3];
  S RS[3][2];          // [s_u t_u, s_v t_v]
  S M[2][2], det;      // M = B_xy R S'
  S Q[2][2], q[2];     // Eq. affine2dgs_Qq
  S c[2];              // projected centre B_xy p + b_xy
  S zc, dzdu, dzdv;    // depth of P(u,v): zc + dzdu u + dzdv v
  S n[3];              // normal, flipped toward the sensor
  double flip;         // +1 / -1
  double ndotv;        // n . v_s before the flip
  bool deg, culled;
  double r2;           // 2 ln(o / alpha_min): alpha >= alpha_min needs |u|^2 <= r2
  double ex, ey;       // conservative half extents of the support in pixels
  S R[3][3];
  double qn[4], qnorm;
};

template <class S>
Proj<S> project(const Scene& sc, const Dirs* dr, int64_t k, const Cam<S>& C, const double* opt) {
  Proj<S> P;
  const int64_t n = sc.n;
  S p[3], sc2[2], qq[4];
  for (int i = 0; i < 3; ++i) p[i] = lift<S>(sc.means[i * n + k], dr ? dr->means : nullptr, i * n + k);
  for (int i = 0; i < 2; ++i) sc2[i] = lift<S>(sc.scales[i * n + k], dr ? dr->scales : nullptr, i * n + k);
  for (int i = 0; i < 4; ++i) qq[i] = lift<S>(sc.quats[i * n + k], dr ? dr->quats : nullptr, i * n + k);
  P.o = lift<S>(sc.opac[k], dr ? dr->opac : nullptr, k);
  for (int i = 0; i < 3; ++i) P.rgb[i] = lift<S>(sc.rgb[i * n + k], dr ? dr->rgb : nullptr, i * n + k);

  // normalised quaternion (w, x, y, z) -> rotation matrix
  S nrm = sqrt(qq[0] * qq[0] + qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3]);
  S w = qq[0] / nrm, x = qq[1] / nrm, y = qq[2] / nrm, z = qq[3] / nrm;
  P.qnorm = val(nrm);
  P.qn[0] = val(w); P.qn[1] = val(x); P.qn[2] = val(y); P.qn[3] = val(z);
  S one(1.0), two(2.0);
  P.R[0][0] = one - two * (y * y + z * z); P.R[0][1] = two * (x * y - w * z); P.R[0][2] = two * (x * z + w * y);
  P.R[1][0] = two * (x * y + w * z); P.R[1][1] = one - two * (x * x + z * z); P.R[1][2] = two * (y * z - w * x);
  P.R[2][0] = two * (x * z - w * y); P.R[2][1] = two * (y * z + w * x); P.R[2][2] = one - two * (x * x + y * y);
  for (int i = 0; i < 3; ++i) {
    P.RS[i][0] = sc2[0] * P.R[i][0];
    P.RS[i][1] = sc2[1] * P.R[i][1];
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      P.M[i][j] = C.B[i][0] * P.RS[0][j] + C.B[i][1] * P.RS[1][j] + C.B[i][2] * P.RS[2][j];
  P.det = P.M[0][0] * P.M[1][1] - P.M[0][1] * P.M[1][0];
  for (int i = 0; i < 2; ++i)
    P.c[i] = C.B[i][0] * p[0] + C.B[i][1] * p[1] + C.B[i][2] * p[2] + C.b[i];
  P.deg = std::fabs(val(P.det)) < opt[O_DETEPS];
  if (!P.deg) {
    P.Q[0][0] = P.M[1][1] / P.det;
    P.Q[0][1] = -P.M[0][1] / P.det;
    P.Q[1][0] = -P.M[1][0] / P.det;
    P.Q[1][1] = P.M[0][0] / P.det;
    for (int i = 0; i < 2; ++i) P.q[i] = -(P.Q[i][0] * P.c[0] + P.Q[i][1] * P.c[1]);
  } else {
    for (int i = 0; i < 2; ++i) { P.Q[i][0] = P.Q[i][1] = S(0.0); P.q[i] = S(0.0); }
  }
  // depth z = B_z P(u,v) + b_z with B_z = [0,0,-1], b_z = max_altitude (Eq. depth_affine_camera)
  P.zc = S(C.maxalt) - p[2];
  P.dzdu = -P.RS[2][0];
  P.dzdv = -P.RS[2][1];
  double nd = val(P.R[0][2]) * C.vs[0] + val(P.R[1][2]) * C.vs[1] + val(P.R[2][2]) * C.vs[2];
  P.ndotv = nd;
  P.flip = nd < 0 ? -1.0 : 1.0;
  for (int i = 0; i < 3; ++i) P.n[i] = S(P.flip) * P.R[i][2];
  double o = val(P.o);
  P.culled = !(o >= opt[O_AMIN]);
  P.r2 = P.culled ? 0.0 : 2.0 * std::log(o / opt[O_AMIN]);
  double r = std::sqrt(std::max(P.r2, 0.0));
  double sig = opt[O_SIGMA];
  double m0 = std::sqrt(val(P.M[0][0]) * val(P.M[0][0]) + val(P.M[0][1]) * val(P.M[0][1]));
  double m1 = std::sqrt(val(P.M[1][0]) * val(P.M[1][0]) + val(P.M[1][1]) * val(P.M[1][1]));
  if (P.deg) m0 = m1 = 0.0;
  // padded so that the binned mode never misses a contributor of the brute mode
  P.ex = r * std::max(m0, sig) * (1 + 1e-6) + 1e-6;
  P.ey = r * std::max(m1, sig) * (1 + 1e-6) + 1e-6;
  return P;
}

// ---------------------------------------------------------------- per pixel evaluation
template <class S> struct Eval {
  S alpha, Ghat, Gu, Gs, u, v;
  bool uwin, clamped;
  double oG;  // o * G^ before the clamp
};

template <class S>
inline Eval<S> evaluate(const Proj<S>& P, double px, double py, const double* opt) {
  Eval<S> E;
  S X(px), Y(py);
  double sig = opt[O_SIGMA];
  S dx = X - P.c[0], dy = Y - P.c[1];
  E.Gs = exp(-(dx * dx + dy * dy) / S(2.0 * sig * sig));
  if (!P.deg) {
    E.u = P.Q[0][0] * X + P.Q[0][1] * Y + P.q[0];
    E.v = P.Q[1][0] * X + P.Q[1][1] * Y + P.q[1];
    E.Gu = exp(S(-0.5) * (E.u * E.u + E.v * E.v));
    E.uwin = val(E.Gu) >= val(E.Gs);
    E.Ghat = E.uwin ? E.Gu : E.Gs;
  } else {
    E.u = E.v = S(0.0);
    E.Gu = S(0.0);
    E.uwin = false;
    E.Ghat = E.Gs;
  }
  S oG = P.o * E.Ghat;
  E.oG = val(oG);
  E.clamped = E.oG > opt[O_AMAX];
  E.alpha = E.clamped ? S(opt[O_AMAX]) : oG;
  return E;
}

inline double relmargin(double a, double b) { return std::fabs(a / b - 1.0); }

// ---------------------------------------------------------------- candidate lists
struct Bins {
  int bw, bh, nbx, nby, x0, y0;
  std::vector<std::vector<int64_t>> lists;  // splats in visibility order
};

// visibility order: stored height p_z descending, ties by smaller splat index (Sec. 3.2)
std::vector<int64_t> visibility_order(const Scene& sc) {
  std::vector<int64_t> ord(sc.n);
  for (int64_t k = 0; k < sc.n; ++k) ord[k] = k;
  const double* pz = sc.means + 2 * sc.n;
  std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) {
    if (pz[a] != pz[b]) return pz[a] > pz[b];
    return a < b;
  });
  return ord;
}

template <class S>
void build_bins(Bins& bins, const std::vector<Proj<S>>& P, const std::vector<int64_t>& ord,
                int x0, int y0, int cw, int ch) {
  bins.bw = 16; bins.bh = 16;
  bins.x0 = x0; bins.y0 = y0;
  bins.nbx = (cw + 15) / 16; bins.nby = (ch + 15) / 16;
  bins.lists.assign((size_t)bins.nbx * bins.nby, {});
  for (int64_t k : ord) {
    const Proj<S>& p = P[k];
    if (p.culled) continue;
    double cx = val(p.c[0]), cy = val(p.c[1]);
    double ilo = std::ceil(cx - p.ex - 0.5), ihi = std::floor(cx + p.ex - 0.5);
    double jlo = std::ceil(cy - p.ey - 0.5), jhi = std::floor(cy + p.ey - 0.5);
    ilo = std::max(ilo, (double)x0); ihi = std::min(ihi, (double)(x0 + cw - 1));
    jlo = std::max(jlo, (double)y0); jhi = std::min(jhi, (double)(y0 + ch - 1));
    if (ilo > ihi || jlo > jhi) continue;
    int bx0 = ((int)ilo - x0) / 16, bx1 = ((int)ihi - x0) / 16;
    int by0 = ((int)jlo - y0) / 16, by1 = ((int)jhi - y0) / 16;
    for (int by = by0; by <= by1; ++by)
      for (int bx = bx0; bx <= bx1; ++bx) bins.lists[(size_t)by * bins.nbx + bx].push_back(k);
  }
}

// ---------------------------------------------------------------- the forward definition
template <class S> struct PixOut {
  S rgb[3], depth, nrm[3], alpha, A[3], dist;
  double T;
  int ncontrib, terminated;
  double mfwd, mbwd;
};

template <class S>
PixOut<S> render_pixel(const std::vector<Proj<S>>& P, const std::vector<int64_t>& cand,
                       int i, int j, const Cam<S>& C, const S* color, const double* opt) {
  PixOut<S> out;
  double px = i + 0.5, py = j + 0.5;
  S T(1.0);
  S A[3] = {S(0.0), S(0.0), S(0.0)}, D(0.0), N[3] = {S(0.0), S(0.0), S(0.0)};
  double mf = 1e300, mb = 1e300;
  out.ncontrib = 0;
  out.terminated = 0;
  std::vector<S> wts, zs;  // weights and intersection depths of the composited splats
  for (int64_t k : cand) {
    const Proj<S>& p = P[k];
    if (p.culled) continue;
    Eval<S> E = evaluate(p, px, py, opt);
    double a = val(E.alpha);
    double ma = relmargin(a, opt[O_AMIN]);
    mf = std::min(mf, ma);
    if (!(a >= opt[O_AMIN])) continue;
    double md = relmargin(std::fabs(val(p.det)), opt[O_DETEPS]);
    mf = std::min(mf, md);
    S Tn = T * (S(1.0) - E.alpha);
    double mt = relmargin(val(Tn), opt[O_TMIN]);
    mf = std::min(mf, mt);
    if (val(Tn) < opt[O_TMIN]) { out.terminated = 1; break; }
    mf = std::min(mf, std::fabs(p.ndotv));
    mb = std::min(mb, relmargin(E.oG, opt[O_AMAX]));
    if (!p.deg) {
      double gu = val(E.Gu), gs = val(E.Gs);
      mb = std::min(mb, std::fabs(gu - gs) / std::max(gu, gs));
    }
    S w = E.alpha * T;
    for (int c = 0; c < 3; ++c) A[c] += w * p.rgb[c];
    S z = p.deg ? p.zc : p.zc + p.dzdu * E.u + p.dzdv * E.v;
    D += w * z;
    for (int c = 0; c < 3; ++c) N[c] += w * p.n[c];
    wts.push_back(w);
    zs.push_back(z);
    T = Tn;
    out.ncontrib++;
  }
  // distortion: every composited pair, the later splat i against each earlier one j
  S dist(0.0);
  for (size_t i = 0; i < wts.size(); ++i)
    for (size_t j = 0; j < i; ++j) dist += S(2.0) * wts[i] * wts[j] * (zs[i] - zs[j]);
  out.dist = dist;
  out.T = val(T);
  out.alpha = S(1.0) - T;
  out.depth = D;
  for (int c = 0; c < 3; ++c) {
    out.nrm[c] = N[c];
    out.A[c] = A[c];
    if (!C.sun) {
      out.rgb[c] = color[4 * c + 0] * A[0] + color[4 * c + 1] * A[1] + color[4 * c + 2] * A[2] +
                   color[4 * c + 3];
    } else {
      out.rgb[c] = S(0.0);
    }
  }
  out.mfwd = mf;
  out.mbwd = std::min(mf, mb);
  return out;
}

template <class S>
std::vector<Proj<S>> project_all(const Scene& sc, const Dirs* dr, const Cam<S>& C, const double* opt) {
  std::vector<Proj<S>> P(sc.n);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < sc.n; ++k) P[k] = project<S>(sc, dr, k, C, opt);
  return P;
}

struct Crop {
  int x0, y0, w, h;
};

template <class S>
void forward_image(const Scene& sc, const Dirs* dr, const double* cam, int sun, const double* color_in,
                   const double* opt, Crop cr, int brute,
                   // outputs (values for double, tangents for dual), each [h][w] or [3][h][w]
                   double* rgb, double* depth, double* nrm, double* alpha, double* Tfin,
                   double* mfwd, double* mbwd, int32_t* ncontrib, int32_t* terminated,
                   double* dist) {
  Cam<S> C = assemble<S>(cam, dr ? dr->dF : nullptr, sun != 0);
  S color[12];
  for (int i = 0; i < 12; ++i) {
    double v = color_in ? color_in[i] : ((i % 4 == i / 4) ? 1.0 : 0.0);
    color[i] = lift<S>(v, dr ? dr->color : nullptr, i);
  }
  std::vector<Proj<S>> P = project_all<S>(sc, dr, C, opt);
  std::vector<int64_t> ord = visibility_order(sc);
  Bins bins;
  if (!brute) build_bins<S>(bins, P, ord, cr.x0, cr.y0, cr.w, cr.h);
  const int64_t hw = (int64_t)cr.w * cr.h;
#pragma omp parallel for schedule(dynamic, 1)
  for (int jj = 0; jj < cr.h; ++jj) {
    for (int ii = 0; ii < cr.w; ++ii) {
      int i = cr.x0 + ii, j = cr.y0 + jj;
      const std::vector<int64_t>& cand =
          brute ? ord : bins.lists[(size_t)(jj / 16) * bins.nbx + (ii / 16)];
      PixOut<S> o = render_pixel<S>(P, cand, i, j, C, color, opt);
      int64_t idx = (int64_t)jj * cr.w + ii;
      auto put = [](double* dst, int64_t at, const S& x) {
        if (!dst) return;
        if constexpr (std::is_same<S, double>::value) dst[at] = x;
        else dst[at] = x.d;
      };
      for (int c = 0; c < 3; ++c) {
        put(rgb, c * hw + idx, o.rgb[c]);
        put(nrm, c * hw + idx, o.nrm[c]);
      }
      put(depth, idx, o.depth);
      put(alpha, idx, o.alpha);
      put(dist, idx, o.dist);
      if (Tfin) Tfin[idx] = o.T;
      if (mfwd) mfwd[idx] = o.mfwd;
      if (mbwd) mbwd[idx] = o.mbwd;
      if (ncontrib) ncontrib[idx] = o.ncontrib;
      if (terminated) terminated[idx] = o.terminated;
    }
  }
}

// ---------------------------------------------------------------- hand-written adjoint
// Per-splat accumulators of d(loss)/d(projected quantities) in the paper's notation.
enum { G_Q = 0, G_q = 4, G_cs = 6, G_o = 8, G_zc = 9, G_du = 10, G_dv = 11, G_rgb = 12, G_n = 15, G_NUM = 18 };

void chain_rule_quat(const double qn[4], double qnorm, const double dR[3][3], double dq_raw[4]) {
  double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
  // partial derivatives of R entries w.r.t. (w, x, y, z) of the normalised quaternion
  double dw = 0, dx = 0, dy = 0, dz = 0;
  // R00 = 1 - 2(y^2 + z^2)
  dy += -4 * y * dR[0][0]; dz += -4 * z * dR[0][0];
  // R01 = 2(xy - wz)
  dx += 2 * y * dR[0][1]; dy += 2 * x * dR[0][1]; dw += -2 * z * dR[0][1]; dz += -2 * w * dR[0][1];
  // R02 = 2(xz + wy)
  dx += 2 * z * dR[0][2]; dz += 2 * x * dR[0][2]; dw += 2 * y * dR[0][2]; dy += 2 * w * dR[0][2];
  // R10 = 2(xy + wz)
  dx += 2 * y * dR[1][0]; dy += 2 * x * dR[1][0]; dw += 2 * z * dR[1][0]; dz += 2 * w * dR[1][0];
  // R11 = 1 - 2(x^2 + z^2)
  dx += -4 * x * dR[1][1]; dz += -4 * z * dR[1][1];
  // R12 = 2(yz - wx)
  dy += 2 * z * dR[1][2]; dz += 2 * y * dR[1][2]; dw += -2 * x * dR[1][2]; dx += -2 * w * dR[1][2];
  // R20 = 2(xz - wy)
  dx += 2 * z * dR[2][0]; dz += 2 * x * dR[2][0]; dw += -2 * y * dR[2][0]; dy += -2 * w * dR[2][0];
  // R21 = 2(yz + wx)
  dy += 2 * z * dR[2][1]; dz += 2 * y * dR[2][1]; dw += 2 * x * dR[2][1]; dx += 2 * w * dR[2][1];
  // R22 = 1 - 2(x^2 + y^2)
  dx += -4 * x * dR[2][2]; dy += -4 * y * dR[2][2];
  double g[4] = {dw, dx, dy, dz};
  // q_n = q / |q|:  dq = (g - q_n (q_n . g)) / |q|
  double dot = g[0] * qn[0] + g[1] * qn[1] + g[2] * qn[2] + g[3] * qn[3];
  for (int i = 0; i < 4; ++i) dq_raw[i] = (g[i] - qn[i] * dot) / qnorm;
}

struct Walk {
  int64_t k;
  double alpha, T, Ghat, Gu, Gs, u, v, z;
  bool uwin, clamped;
};

void backward_image(const Scene& sc, const double* cam, int sun, const double* color, const double* opt,
                    Crop cr, int brute,
                    const double* g_rgb, const double* g_depth, const double* g_nrm, const double* g_alpha,
                    const double* g_dist, double* d_means, double* d_scales, double* d_quats, double* d_opac, double* d_rgb,
                    double* d_dF, double* d_color) {
  Cam<double> C = assemble<double>(cam, nullptr, sun != 0);
  double col[12];
  for (int i = 0; i < 12; ++i) col[i] = color ? color[i] : ((i % 4 == i / 4) ? 1.0 : 0.0);
  std::vector<Proj<double>> P = project_all<double>(sc, nullptr, C, opt);
  std::vector<int64_t> ord = visibility_order(sc);
  Bins bins;
  if (!brute) build_bins<double>(bins, P, ord, cr.x0, cr.y0, cr.w, cr.h);
  const int64_t hw = (int64_t)cr.w * cr.h;
  std::vector<double> acc((size_t)sc.n * G_NUM, 0.0);
  double dcol[12] = {0};

#pragma omp parallel
  {
    double dcol_l[12] = {0};
    std::vector<Walk> walk;
#pragma omp for schedule(dynamic, 1)
    for (int jj = 0; jj < cr.h; ++jj) {
      for (int ii = 0; ii < cr.w; ++ii) {
        int i = cr.x0 + ii, j = cr.y0 + jj;
        int64_t idx = (int64_t)jj * cr.w + ii;
        double px = i + 0.5, py = j + 0.5;
        const std::vector<int64_t>& cand =
            brute ? ord : bins.lists[(size_t)(jj / 16) * bins.nbx + (ii / 16)];
        // forward walk, recorded
        walk.clear();
        double T = 1.0, A[3] = {0, 0, 0};
        for (int64_t k : cand) {
          const Proj<double>& p = P[k];
          if (p.culled) continue;
          Eval<double> E = evaluate(p, px, py, opt);
          if (!(E.alpha >= opt[O_AMIN])) continue;
          double Tn = T * (1.0 - E.alpha);
          if (Tn < opt[O_TMIN]) break;
          Walk wk;
          wk.k = k; wk.alpha = E.alpha; wk.T = T; wk.Ghat = E.Ghat; wk.Gu = E.Gu; wk.Gs = E.Gs;
          wk.u = E.u; wk.v = E.v; wk.uwin = E.uwin; wk.clamped = E.clamped;
          wk.z = p.deg ? p.zc : p.zc + p.dzdu * E.u + p.dzdv * E.v;
          walk.push_back(wk);
          double w = E.alpha * T;
          for (int c = 0; c < 3; ++c) A[c] += w * p.rgb[c];
          T = Tn;
        }
        const double Tfinal = T;
        // upstream of the pixel
        double gA[3] = {0, 0, 0}, gN[3] = {0, 0, 0}, gD = 0, gAl = 0;
        if (!sun && g_rgb) {
          double gr[3] = {g_rgb[idx], g_rgb[hw + idx], g_rgb[2 * hw + idx]};
          // rgb_out = C A + c  ->  dA = C^T g, dC = g A^T, dc = g
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) gA[b] += col[4 * a + b] * gr[a];
          for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b) dcol_l[4 * a + b] += gr[a] * A[b];
            dcol_l[4 * a + 3] += gr[a];
          }
        }
        if (!sun && g_nrm)
          for (int c = 0; c < 3; ++c) gN[c] = g_nrm[c * hw + idx];
        if (g_depth) gD = g_depth[idx];
        if (g_alpha) gAl = g_alpha[idx];
        // distortion: its partials in the weight and in the depth of each composited splat m,
        // as plain sums over the other composited splats:
        //   d/dw_m = sum_{j<m} 2 w_j (z_m - z_j) + sum_{i>m} 2 w_i (z_i - z_m)
        //   d/dz_m = sum_{j<m} 2 w_m w_j - sum_{i>m} 2 w_i w_m
        const double gDist = g_dist ? g_dist[idx] : 0.0;
        const size_t nw = walk.size();
        std::vector<double> hw(nw, 0.0), hz(nw, 0.0);
        if (gDist != 0.0) {
          for (size_t m = 0; m < nw; ++m) {
            const double wm = walk[m].alpha * walk[m].T, zm = walk[m].z;
            for (size_t j = 0; j < nw; ++j) {
              if (j == m) continue;
              const double wj = walk[j].alpha * walk[j].T, zj = walk[j].z;
              if (j < m) {
                hw[m] += 2.0 * wj * (zm - zj);
                hz[m] += 2.0 * wm * wj;
              } else {
                hw[m] += 2.0 * wj * (zj - zm);
                hz[m] -= 2.0 * wj * wm;
              }
            }
          }
        }
        // reverse walk: f = sum_i f_i a_i T_i, T_i = prod_{j<i} (1 - a_j);
        // df/da_i = T_i (f_i - S_i), S_i = sum_{j>i} f_j a_j prod_{i<l<j} (1 - a_l)
        double Sg = 0.0;  // g . S_i
        for (int m = (int)walk.size() - 1; m >= 0; --m) {
          const Walk& wk = walk[m];
          const Proj<double>& p = P[wk.k];
          double w = wk.alpha * wk.T;
          double gf = gD * wk.z + gDist * hw[m];
          for (int c = 0; c < 3; ++c) gf += gA[c] * p.rgb[c] + gN[c] * p.n[c];
          double dalpha = wk.T * (gf - Sg) + gAl * Tfinal / (1.0 - wk.alpha);
          Sg = wk.alpha * gf + (1.0 - wk.alpha) * Sg;
          double g[G_NUM] = {0};
          for (int c = 0; c < 3; ++c) {
            g[G_rgb + c] = w * gA[c];
            g[G_n + c] = w * gN[c];
          }
          double dz = w * gD + gDist * hz[m];
          double du = 0, dv = 0;
          g[G_zc] = dz;
          if (!p.deg) {
            g[G_du] = dz * wk.u;
            g[G_dv] = dz * wk.v;
            du += dz * p.dzdu;
            dv += dz * p.dzdv;
          }
          if (!wk.clamped) {
            g[G_o] = dalpha * wk.Ghat;
            double dG = dalpha * p.o;
            if (wk.uwin) {
              // G = exp(-(u^2 + v^2)/2)
              du += -dG * wk.Gu * wk.u;
              dv += -dG * wk.Gu * wk.v;
            } else {
              // G = exp(-|x - c|^2 / (2 sigma^2))
              double s2 = opt[O_SIGMA] * opt[O_SIGMA];
              double fx = px - p.c[0], fy = py - p.c[1];
              g[G_cs + 0] = dG * wk.Gs * fx / s2;
              g[G_cs + 1] = dG * wk.Gs * fy / s2;
            }
          }
          if (!p.deg) {
            // u = Q x + q
            g[G_Q + 0] = du * px; g[G_Q + 1] = du * py;
            g[G_Q + 2] = dv * px; g[G_Q + 3] = dv * py;
            g[G_q + 0] = du; g[G_q + 1] = dv;
          }
          double* a = &acc[(size_t)wk.k * G_NUM];
          for (int f = 0; f < G_NUM; ++f) {
            if (g[f] != 0.0) {
#pragma omp atomic
              a[f] += g[f];
            }
          }
        }
      }
    }
#pragma omp critical
    for (int i = 0; i < 12; ++i) dcol[i] += dcol_l[i];
  }
  if (d_color && !sun)
    for (int i = 0; i < 12; ++i) d_color[i] += dcol[i];

  // chain the per-splat accumulators through the projection (per splat, then the camera)
  double dB[2][3] = {{0}}, db[2] = {0};
  const int64_t n = sc.n;
  for (int64_t k = 0; k < n; ++k) {
    const Proj<double>& p = P[k];
    const double* g = &acc[(size_t)k * G_NUM];
    bool any = false;
    for (int f = 0; f < G_NUM; ++f) any |= (g[f] != 0.0);
    if (!any || p.culled) continue;
    double pm[3] = {sc.means[k], sc.means[n + k], sc.means[2 * n + k]};
    double su = sc.scales[k], sv = sc.scales[n + k];
    double dQ[2][2] = {{g[G_Q + 0], g[G_Q + 1]}, {g[G_Q + 2], g[G_Q + 3]}};
    double dq[2] = {g[G_q + 0], g[G_q + 1]};
    double dc[2] = {g[G_cs + 0], g[G_cs + 1]};
    double dM[2][2] = {{0, 0}, {0, 0}};
    if (!p.deg) {
      // q = -Q c
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          dQ[a][b] += -dq[a] * p.c[b];
          dc[b] += -p.Q[a][b] * dq[a];
        }
      // Q = M^-1:  dM = -Q^T dQ Q^T
      double t[2][2];
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) t[a][b] = p.Q[0][a] * dQ[0][b] + p.Q[1][a] * dQ[1][b];
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) dM[a][b] = -(t[a][0] * p.Q[b][0] + t[a][1] * p.Q[b][1]);
    }
    // c = B p + b
    double dp[3] = {0, 0, 0};
    for (int a = 0; a < 2; ++a) {
      for (int b = 0; b < 3; ++b) {
        dB[a][b] += dc[a] * pm[b];
        dp[b] += C.B[a][b] * dc[a];
      }
      db[a] += dc[a];
    }
    // M = B RS'
    double dRS[3][2] = {{0}};
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 3; ++b) {
        dB[a][b] += dM[a][0] * p.RS[b][0] + dM[a][1] * p.RS[b][1];
        for (int e = 0; e < 2; ++e) dRS[b][e] += C.B[a][b] * dM[a][e];
      }
    // depth: zc = max_alt - p_z; dzdu = -s_u R20, dzdv = -s_v R21
    dp[2] += -g[G_zc];
    double dR[3][3] = {{0}};
    double dsu = 0, dsv = 0;
    dsu += -g[G_du] * p.R[2][0];
    dR[2][0] += -g[G_du] * su;
    dsv += -g[G_dv] * p.R[2][1];
    dR[2][1] += -g[G_dv] * sv;
    // RS' = [s_u R[:,0], s_v R[:,1]]
    for (int b = 0; b < 3; ++b) {
      dsu += dRS[b][0] * p.R[b][0];
      dsv += dRS[b][1] * p.R[b][1];
      dR[b][0] += dRS[b][0] * su;
      dR[b][1] += dRS[b][1] * sv;
    }
    // normal = flip * R[:,2]
    for (int b = 0; b < 3; ++b) dR[b][2] += p.flip * g[G_n + b];
    double dqr[4];
    chain_rule_quat(p.qn, p.qnorm, dR, dqr);
    for (int b = 0; b < 3; ++b) d_means[b * n + k] += dp[b];
    d_scales[k] += dsu;
    d_scales[n + k] += dsv;
    for (int b = 0; b < 4; ++b) d_quats[b * n + k] += dqr[b];
    d_opac[k] += g[G_o];
    for (int b = 0; b < 3; ++b) d_rgb[b * n + k] += g[G_rgb + b];
  }
  // camera: main B = F_B + dF_B; sun B_sun = S B' (I - s e3^T), b_sun = S b'
  double dBp[2][3], dbp[2];
  if (!sun) {
    for (int a = 0; a < 2; ++a) {
      for (int b = 0; b < 3; ++b) dBp[a][b] = dB[a][b];
      dbp[a] = db[a];
    }
  } else {
    for (int a = 0; a < 2; ++a) {
      for (int k2 = 0; k2 < 3; ++k2) {
        double s = 0;
        for (int j2 = 0; j2 < 3; ++j2) {
          double Pkj = (k2 == j2 ? 1.0 : 0.0) - (j2 == 2 ? C.s[k2] : 0.0);
          s += dB[a][j2] * Pkj;
        }
        dBp[a][k2] = C.S_ * s;
      }
      dbp[a] = C.S_ * db[a];
    }
  }
  if (d_dF)
    for (int a = 0; a < 2; ++a) {
      for (int b = 0; b < 3; ++b) d_dF[4 * a + b] += dBp[a][b];
      d_dF[4 * a + 3] += dbp[a];
    }
}

Scene make_scene(int64_t n, const double* means, const double* scales, const double* quats,
                 const double* opac, const double* rgb) {
  Scene s;
  s.n = n; s.means = means; s.scales = scales; s.quats = quats; s.opac = opac; s.rgb = rgb;
  return s;
}

}  // namespace

extern "C" {

int ora_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void ora_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* Assembled camera: B (2x3 row-major), b (2), unit view direction toward the sensor (3),
 * image width/height. */
void ora_camera(const double* cam, int sun, double* B, double* b, double* vs, int* wh) {
  Cam<double> C = assemble<double>(cam, nullptr, sun != 0);
  for (int i = 0; i < 2; ++i) {
    for (int j = 0; j < 3; ++j) B[3 * i + j] = C.B[i][j];
    b[i] = C.b[i];
  }
  for (int i = 0; i < 3; ++i) vs[i] = C.vs[i];
  wh[0] = C.W; wh[1] = C.H;
}

/* Per-splat projected quantities, 24 doubles per splat:
 * M(4) det Q(4) q(2) c(2) zc dzdu dzdv n(3) r2 ex ey deg culled */
void ora_project(int64_t n, const double* means, const double* scales, const double* quats,
                 const double* opac, const double* rgb, const double* cam, int sun, const double* opt,
                 double* out) {
  Scene sc = make_scene(n, means, scales, quats, opac, rgb);
  Cam<double> C = assemble<double>(cam, nullptr, sun != 0);
  for (int64_t k = 0; k < n; ++k) {
    Proj<double> p = project<double>(sc, nullptr, k, C, opt);
    double* o = out + 24 * k;
    o[0] = p.M[0][0]; o[1] = p.M[0][1]; o[2] = p.M[1][0]; o[3] = p.M[1][1]; o[4] = p.det;
    o[5] = p.Q[0][0]; o[6] = p.Q[0][1]; o[7] = p.Q[1][0]; o[8] = p.Q[1][1];
    o[9] = p.q[0]; o[10] = p.q[1]; o[11] = p.c[0]; o[12] = p.c[1];
    o[13] = p.zc; o[14] = p.dzdu; o[15] = p.dzdv;
    o[16] = p.n[0]; o[17] = p.n[1]; o[18] = p.n[2];
    o[19] = p.r2; o[20] = p.ex; o[21] = p.ey; o[22] = p.deg ? 1 : 0; o[23] = p.culled ? 1 : 0;
  }
}

/* Visibility order (splat indices front to back). */
void ora_order(int64_t n, const double* means, int64_t* order) {
  Scene sc = make_scene(n, means, nullptr, nullptr, nullptr, nullptr);
  std::vector<int64_t> o = visibility_order(sc);
  std::memcpy(order, o.data(), sizeof(int64_t) * n);
}

/* Forward render of the crop (x0, y0, w, h) of one view (sun = 0) or its sun view (sun = 1).
 * Outputs are planar [C][h][w]; any output pointer may be NULL.  o_dist is the distortion
 * of the pixel's blending weights (see the header). */
void ora_render(int64_t n, const double* means, const double* scales, const double* quats,
                const double* opac, const double* rgb, const double* cam, int sun,
                const double* color, const double* opt, int x0, int y0, int w, int h, int brute,
                double* o_rgb, double* o_depth, double* o_nrm, double* o_alpha, double* o_T,
                double* o_mfwd, double* o_mbwd, int32_t* o_ncontrib, int32_t* o_term, double* o_dist) {
  Scene sc = make_scene(n, means, scales, quats, opac, rgb);
  forward_image<double>(sc, nullptr, cam, sun, color, opt, Crop{x0, y0, w, h}, brute, o_rgb, o_depth,
                        o_nrm, o_alpha, o_T, o_mfwd, o_mbwd, o_ncontrib, o_term, o_dist);
}

/* Directional derivative (forward mode, dual numbers) of the rendered planes along the
 * given tangent of every input (any direction pointer may be NULL = 0). */
void ora_render_dual(int64_t n, const double* means, const double* scales, const double* quats,
                     const double* opac, const double* rgb, const double* cam, int sun,
                     const double* color, const double* opt, int x0, int y0, int w, int h, int brute,
                     const double* t_means, const double* t_scales, const double* t_quats,
                     const double* t_opac, const double* t_rgb, const double* t_dF, const double* t_color,
                     double* o_rgb, double* o_depth, double* o_nrm, double* o_alpha, double* o_dist) {
  Scene sc = make_scene(n, means, scales, quats, opac, rgb);
  Dirs d{t_means, t_scales, t_quats, t_opac, t_rgb, t_dF, t_color};
  forward_image<Dual>(sc, &d, cam, sun, color, opt, Crop{x0, y0, w, h}, brute, o_rgb, o_depth, o_nrm,
                      o_alpha, nullptr, nullptr, nullptr, nullptr, nullptr, o_dist);
}

/* Reverse-mode adjoint of the crop's planes: gradients are ADDED into the outputs.
 * Upstream planes are [C][h][w] over the crop (NULL = 0); g_dist is the upstream of the
 * distortion plane. */
void ora_backward(int64_t n, const double* means, const double* scales, const double* quats,
                  const double* opac, const double* rgb, const double* cam, int sun,
                  const double* color, const double* opt, int x0, int y0, int w, int h, int brute,
                  const double* g_rgb, const double* g_depth, const double* g_nrm, const double* g_alpha,
                  const double* g_dist, double* d_means, double* d_scales, double* d_quats, double* d_opac,
                  double* d_rgb, double* d_dF, double* d_color) {
  Scene sc = make_scene(n, means, scales, quats, opac, rgb);
  backward_image(sc, cam, sun, color, opt, Crop{x0, y0, w, h}, brute, g_rgb, g_depth, g_nrm, g_alpha,
                 g_dist, d_means, d_scales, d_quats, d_opac, d_rgb, d_dF, d_color);
}

}  // extern "C"
