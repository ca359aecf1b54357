// CPU oracle for the voxel ray-tracing path of "Real-Time Rendering of Dynamic
// Line Sets using Voxel Ray Tracing" (Kraaijeveld et al., arXiv 2510.09081).
//
// TEST INFRASTRUCTURE ONLY. This file is plain, slow, obviously-correct C++17
// that restates the paper's definitions in fp64 (and exact integer arithmetic
// where a geometric predicate decides an integer result). Only the tests, the
// smoke check and the benchmark's CPU-baseline leg may load it; the product
// path never does. It shares no code with the CUDA library.
//
// What it computes, in the paper's order:
//   * ingest     -- vertices snapped to multiples of 2^-14 voxel; per-vertex
//                   first/last flags; clip-plane normals as central-difference
//                   tangents (Sec. 3.1, after Gross & Gumhold), disabled at
//                   polyline ends.
//   * lists      -- per-voxel segment lists: segment i (vertex i -> i+1, Sec. 3.3)
//                   is listed in voxel v iff the closed distance between the
//                   segment and v's closed box is <= the list radius
//                   (conservative capsule voxelization, Sec. 3.1). Decided
//                   exactly in integers. Lists are sorted by segment id.
//   * occupancy  -- Alg. 3 (PWAA-clamped clipped-capsule SDF of Alg. 2) sampled
//                   at the voxel centre, quantized per contribution and summed
//                   (Sec. 3.1, packed 16-bit occupancy).
//   * mips       -- averaging occupancy pyramid (Sec. 3.1).
//   * render     -- every hit of every listed segment along each pixel ray, the
//                   first entry into the capsule kept when the clip planes keep
//                   it, sorted by (t, id) and composited front to back
//                   (ground-truth transparency, Sec. 3.5); optional cone-traced
//                   ambient occlusion per hit (Sec. 3.4 cones over the occupancy
//                   pyramid), or voxel-space shading (Sec. 3.4): ambient
//                   occlusion and a directional shadow evaluated at voxel
//                   centres, sampled trilinearly at each hit.
//   * brute      -- the same image from all segments, no lists (pin for the
//                   conservativeness claim of Sec. 3.5).
//   * sampled    -- one voxel's fragments (list and occupancy codes) and a list
//                   of pixels, both by brute force over every segment, for
//                   sampled checks of sets too large for a full list build.
//
// Parity bookkeeping: where an fp32 implementation could legitimately take the
// other side of a near-tie (a grazing ray, a hit on a clip plane or the grid
// boundary, two hits at nearly the same depth, an occupancy code on a rounding
// boundary), the oracle records the alternative result next to the primary one.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <unordered_set>
#include <vector>

namespace {

typedef __int128 i128;

const int64_t UNITS = 16384;            // coordinate units per voxel (2^14)
const int64_t LIST_MARGIN_UNITS = 32;   // list radius = r + 2^-9 voxel
const double T_STOP = 1e-4;             // transmittance where compositing may stop

// ------------------------------------------------------------------ helpers
struct V3 { double x, y, z; };
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 normalize(V3 a) { return (1.0 / norm(a)) * a; }
inline double comp(V3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

template <class F>
void parallel_for(int64_t n, int nthreads, F fn, int64_t chunk = 64) {
  if (nthreads <= 1 || n < 2) {
    for (int64_t i = 0; i < n; ++i) fn(i);
    return;
  }
  std::atomic<int64_t> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&]() {
      for (;;) {
        int64_t b = next.fetch_add(chunk);
        if (b >= n) break;
        int64_t e = std::min(n, b + chunk);
        for (int64_t i = b; i < e; ++i) fn(i);
      }
    });
  for (auto& t : th) t.join();
}

// ------------------------------------------------- exact segment-box predicate
// Is there a point of segment [A, B] within distance R of the closed box
// [lo, lo + S]^3? All inputs are integers (units of 2^-14 voxel).
//
// The set of points within R of the box is the union of
//   (a) three boxes: the box grown by R along one axis only,
//   (b) twelve edge cylinders of radius R, each cut to the slab of its edge,
//   (c) eight corner balls of radius R.
// (A point outside the box along k axes is within R of it exactly when it lies
// in the piece for that k: a face slab for k <= 1, an edge cylinder for k = 2,
// a corner ball for k = 3.) The segment meets the union iff it meets a piece;
// each piece test is exact in 128-bit integers.

struct Frac { i128 n, d; };  // n / d, d > 0
inline bool frac_le(Frac a, Frac b) { return a.n * b.d <= b.n * a.d; }

// t-interval of the segment inside lo_k <= A_k + t D_k <= hi_k, for t in [lo, hi].
// Returns false if empty.
bool clip_axis(int64_t A, int64_t D, int64_t lo, int64_t hi, Frac& tlo, Frac& thi) {
  if (D == 0) return A >= lo && A <= hi;
  Frac a, b;
  if (D > 0) { a = {(i128)(lo - A), (i128)D}; b = {(i128)(hi - A), (i128)D}; }
  else       { a = {(i128)(A - hi), (i128)(-D)}; b = {(i128)(A - lo), (i128)(-D)}; }
  if (frac_le(tlo, a)) tlo = a;
  if (frac_le(b, thi)) thi = b;
  return frac_le(tlo, thi);
}

bool seg_meets_box(const int64_t A[3], const int64_t D[3], const int64_t lo[3],
                   const int64_t hi[3]) {
  Frac tlo = {0, 1}, thi = {1, 1};
  for (int k = 0; k < 3; ++k)
    if (!clip_axis(A[k], D[k], lo[k], hi[k], tlo, thi)) return false;
  return true;
}

// min over t in [tlo, thi] of |W + t E|^2 <= R^2, W, E in 2D or 3D.
bool quad_min_le(const i128* W, const i128* E, int dim, Frac tlo, Frac thi, i128 R2) {
  i128 EE = 0, WE = 0, WW = 0;
  for (int k = 0; k < dim; ++k) { EE += E[k] * E[k]; WE += W[k] * E[k]; WW += W[k] * W[k]; }
  if (EE == 0) return WW <= R2;
  Frac ts = {-WE, EE};  // unconstrained minimiser
  if (frac_le(tlo, ts) && frac_le(ts, thi)) {
    // minimum value = (|W|^2 |E|^2 - (W.E)^2) / |E|^2 = |W x E|^2 / |E|^2
    i128 c2;
    if (dim == 2) {
      i128 c = W[0] * E[1] - W[1] * E[0];
      c2 = c * c;
    } else {
      i128 cx = W[1] * E[2] - W[2] * E[1];
      i128 cy = W[2] * E[0] - W[0] * E[2];
      i128 cz = W[0] * E[1] - W[1] * E[0];
      c2 = cx * cx + cy * cy + cz * cz;
    }
    return c2 <= R2 * EE;
  }
  // convex: the minimum over the interval is at an end point
  for (int e = 0; e < 2; ++e) {
    Frac t = e ? thi : tlo;
    i128 s = 0;
    for (int k = 0; k < dim; ++k) {
      i128 v = W[k] * t.d + t.n * E[k];
      s += v * v;
    }
    if (s <= R2 * t.d * t.d) return true;
  }
  return false;
}

bool seg_box_within(const int64_t A[3], const int64_t B[3], const int64_t lo[3], int64_t S,
                    int64_t R) {
  int64_t D[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
  int64_t hi[3] = {lo[0] + S, lo[1] + S, lo[2] + S};
  const i128 R2 = (i128)R * R;
  // (a) face slabs
  for (int k = 0; k < 3; ++k) {
    int64_t l2[3] = {lo[0], lo[1], lo[2]}, h2[3] = {hi[0], hi[1], hi[2]};
    l2[k] -= R; h2[k] += R;
    if (seg_meets_box(A, D, l2, h2)) return true;
  }
  // (b) edge cylinders: edge along axis m at corner coordinates (ck, cl)
  for (int m = 0; m < 3; ++m) {
    int k = (m + 1) % 3, l = (m + 2) % 3;
    Frac tlo = {0, 1}, thi = {1, 1};
    if (!clip_axis(A[m], D[m], lo[m], hi[m], tlo, thi)) continue;
    for (int ek = 0; ek < 2; ++ek)
      for (int el = 0; el < 2; ++el) {
        int64_t ck = ek ? hi[k] : lo[k], cl = el ? hi[l] : lo[l];
        i128 W[2] = {(i128)(A[k] - ck), (i128)(A[l] - cl)};
        i128 E[2] = {(i128)D[k], (i128)D[l]};
        if (quad_min_le(W, E, 2, tlo, thi, R2)) return true;
      }
  }
  // (c) corner balls
  for (int c = 0; c < 8; ++c) {
    i128 W[3], E[3];
    for (int k = 0; k < 3; ++k) {
      int64_t ck = ((c >> k) & 1) ? hi[k] : lo[k];
      W[k] = (i128)(A[k] - ck);
      E[k] = (i128)D[k];
    }
    if (quad_min_le(W, E, 3, Frac{0, 1}, Frac{1, 1}, R2)) return true;
  }
  return false;
}

inline int64_t floordiv(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

// --------------------------------------------------- Alg. 2 and Alg. 3 (fp64)
// Signed distance from p to the capsule (v0, v1, r) cut by the planes through v0
// (normal n0, keeps the side n0 points to) and v1 (normal n1, keeps the side
// opposite to n1). A disabled plane drops its term from the max.
double clipped_capsule_sdf(V3 p, V3 v0, V3 v1, V3 n0, V3 n1, int en0, int en1, double r) {
  V3 d = v1 - v0;
  V3 pv0 = p - v0, pv1 = p - v1;
  double dd = dot(d, d);
  double h = dd > 0 ? std::min(1.0, std::max(0.0, dot(pv0, d) / dd)) : 0.0;
  double s = norm(pv0 - h * d) - r;
  if (en0) s = std::max(s, -dot(pv0, n0));
  if (en1) s = std::max(s, dot(pv1, n1));
  return s;
}

double capsule_occupancy(V3 p, V3 v0, V3 v1, V3 n0, V3 n1, int en0, int en1, double r,
                         double r_min) {
  double rc = std::max(r, r_min);
  double corr = (r / rc) * (r / rc);
  double sdf = clipped_capsule_sdf(p, v0, v1, n0, n1, en0, en1, rc);
  double occ = std::min(1.0, std::max(0.0, 0.5 - sdf));
  return occ * corr;
}

// ------------------------------------------------------------ ray and capsule
struct Hit {
  double t;     // entry parameter (finite if the line meets the capsule)
  double disc;  // discriminant / r^2 of the piece that gave the entry
};

// First entry of the line o + t d (|d| = 1) into the capsule (a, b, r): the
// smallest entry parameter over its three convex pieces (two balls and the
// finite cylinder). A flat end of the finite cylinder lies inside a ball, so the
// cylinder only contributes entries through its curved side. Returns t = +inf
// when the line misses. `near_disc` receives the smallest |discriminant| / r^2
// over the parts of the pieces that form the capsule's surface (grazing
// bookkeeping for parity).
Hit line_capsule_entry(V3 o, V3 d, V3 a, V3 b, double r, double* near_disc) {
  Hit best = {INFINITY, 0.0};
  double nd = INFINITY;
  const double r2 = r * r;
  V3 ba = b - a;
  double L2 = dot(ba, ba);
  double L = std::sqrt(L2);
  for (int e = 0; e < 2; ++e) {  // balls
    V3 c = e ? b : a;
    V3 oc = o - c;
    double bq = dot(oc, d);
    V3 w = oc - bq * d;
    double ww = dot(w, w);
    double disc = r2 - ww;
    // the silhouette point of the ball nearest the line is on the capsule's
    // surface only on the ball's outer cap
    bool outer = true;
    if (L2 > 0 && ww > 0) {
      V3 contact = c + (r / std::sqrt(ww)) * w;
      double y = dot(contact - a, ba) / L;
      outer = e ? (y >= L) : (y <= 0);
    }
    if (outer) nd = std::min(nd, std::fabs(disc) / r2);
    if (disc < 0) continue;
    double t = -bq - std::sqrt(disc);
    if (t < best.t) best = {t, disc / r2};
  }
  if (L2 > 0) {
    V3 u = (1.0 / L) * ba;
    V3 oa = o - a;
    V3 dp = d - dot(d, u) * u;
    V3 op = oa - dot(oa, u) * u;
    double A = dot(dp, dp);
    if (A > 0) {
      double ts = -dot(op, dp) / A;
      V3 w = op + ts * dp;
      double disc = r2 - dot(w, w);
      double t = disc >= 0 ? ts - std::sqrt(disc / A) : ts;
      double y = dot(oa + t * d, u);
      if (y >= 0 && y <= L) {
        nd = std::min(nd, std::fabs(disc) / r2);
        if (disc >= 0 && t < best.t) best = {t, disc / r2};
      }
    }
  }
  if (near_disc) *near_disc = nd;
  return best;
}

// ------------------------------------------------------------------- context
struct Camera {
  int width, height, ortho;
  double eye[3], target[3], up[3], fovy_deg, ortho_h;
};
// Parity bands: how close to its threshold an fp32 decision may sit before the
// oracle also accepts the other outcome.
struct Params {
  double alpha;
  int ao_cones;
  int voxel_shading;         // 1: shade from the voxel-space shading field
  V3 light;                  // unit direction toward the light (voxel shading)
  double tie_rel, tie_abs;   // two depths tie if |ta - tb| <= tie_abs + tie_rel * max(|t|)
  double graze_rel;          // a ray grazes if |discriminant| / r^2 <= graze_rel
  double pos_abs, pos_rel;   // a hit point is within pos_abs + pos_rel * t of a clip
                             // plane or the grid boundary
};

struct Ctx {
  int N = 0;
  int64_t V = 0, P = 0;
  int64_t R = 0, RL = 0;     // render radius and list radius, units
  double r = 0, r_min = 0.5;
  int Q = 32;                // occupancy codes per unit occupancy
  int nthreads = 1;
  int status = 0;
  std::vector<int64_t> X;    // snapped units, 3 per vertex
  std::vector<V3> pos;       // snapped, voxel units
  std::vector<V3> nrm;
  std::vector<uint8_t> en;   // clip plane enabled
  std::vector<uint8_t> first, last;
  // lists (CSR over canonical voxel index (z*N + y)*N + x)
  std::vector<uint64_t> start;
  std::vector<uint32_t> ids;
  std::vector<uint32_t> occ_nom, occ_lo, occ_hi;
  std::vector<double> mips;  // level 0 .. log2 N, concatenated
  std::vector<int64_t> level_off;
  bool have_lists = false, have_mips = false;
  int64_t F_ambiguous = 0;   // occupancy contributions on a rounding boundary
};

inline bool seg_valid(const Ctx& c, int64_t i) { return i + 1 < c.V && !c.last[i]; }

// ------------------------------------------------------------ list building
// Voxel range [vlo, vhi] (clamped) that can hold voxels within r_L of segment i.
void seg_voxel_range(const Ctx& c, int64_t i, int64_t* vlo, int64_t* vhi) {
  const int64_t* A = &c.X[3 * i];
  const int64_t* B = &c.X[3 * (i + 1)];
  for (int k = 0; k < 3; ++k) {
    int64_t mn = std::min(A[k], B[k]) - c.RL, mx = std::max(A[k], B[k]) + c.RL;
    vlo[k] = std::max<int64_t>(0, floordiv(mn, UNITS) - 1);
    vhi[k] = std::min<int64_t>(c.N - 1, floordiv(mx, UNITS));
  }
}

// Is voxel (x, y, z) within r_L of segment i (exact)? If so, its occupancy code
// (Alg. 2/3 at the voxel centre, rounded to Q codes) and, where Q * occupancy
// lies within 1e-3 of a rounding boundary, both neighbouring codes.
bool fragment(const Ctx& c, int64_t i, int64_t x, int64_t y, int64_t z, uint32_t& qn,
              uint32_t& ql, uint32_t& qh, bool& ambiguous) {
  const int64_t lo[3] = {x * UNITS, y * UNITS, z * UNITS};
  if (!seg_box_within(&c.X[3 * i], &c.X[3 * (i + 1)], lo, UNITS, c.RL)) return false;
  V3 p = {x + 0.5, y + 0.5, z + 0.5};
  double occ = capsule_occupancy(p, c.pos[i], c.pos[i + 1], c.nrm[i], c.nrm[i + 1], c.en[i],
                                 c.en[i + 1], c.r, c.r_min);
  double xq = (double)c.Q * occ;
  double fl = std::floor(xq);
  double fr = xq - fl;
  qn = (uint32_t)std::floor(xq + 0.5);
  ql = qn; qh = qn;
  ambiguous = std::fabs(fr - 0.5) < 1e-3;
  if (ambiguous) { ql = (uint32_t)fl; qh = (uint32_t)fl + 1; }
  return true;
}

void build_lists(Ctx& c) {
  const int N = c.N;
  const int64_t nv = (int64_t)N * N * N;
  // fragments per segment: voxel indices and occupancy codes
  struct SegOut { std::vector<uint32_t> vox; std::vector<uint32_t> qlo, qhi, qnom; };
  std::vector<SegOut> out(c.V);
  std::atomic<int64_t> amb(0);
  parallel_for(c.V, c.nthreads, [&](int64_t i) {
    if (!seg_valid(c, i)) return;
    int64_t vlo[3], vhi[3];
    seg_voxel_range(c, i, vlo, vhi);
    SegOut& so = out[i];
    for (int64_t z = vlo[2]; z <= vhi[2]; ++z)
      for (int64_t y = vlo[1]; y <= vhi[1]; ++y)
        for (int64_t x = vlo[0]; x <= vhi[0]; ++x) {
          uint32_t qn, ql, qh;
          bool a;
          if (!fragment(c, i, x, y, z, qn, ql, qh, a)) continue;
          if (a) amb++;
          so.vox.push_back((uint32_t)((z * N + y) * N + x));
          so.qnom.push_back(qn); so.qlo.push_back(ql); so.qhi.push_back(qh);
        }
  });
  c.F_ambiguous = amb.load();
  std::vector<uint64_t> cnt(nv, 0);
  c.occ_nom.assign(nv, 0); c.occ_lo.assign(nv, 0); c.occ_hi.assign(nv, 0);
  for (int64_t i = 0; i < c.V; ++i)
    for (size_t j = 0; j < out[i].vox.size(); ++j) {
      uint32_t v = out[i].vox[j];
      cnt[v]++;
      c.occ_nom[v] += out[i].qnom[j];
      c.occ_lo[v] += out[i].qlo[j];
      c.occ_hi[v] += out[i].qhi[j];
    }
  c.start.assign(nv + 1, 0);
  for (int64_t v = 0; v < nv; ++v) c.start[v + 1] = c.start[v] + cnt[v];
  c.ids.assign(c.start[nv], 0);
  std::vector<uint64_t> cur(c.start.begin(), c.start.end() - 1);
  // segments visited in increasing id order, so every list comes out sorted
  for (int64_t i = 0; i < c.V; ++i)
    for (uint32_t v : out[i].vox) c.ids[cur[v]++] = (uint32_t)i;
  c.have_lists = true;
}

// --------------------------------------------------------------------- mips
void build_mips(Ctx& c) {
  const int N = c.N;
  int L = 0;
  while ((1 << L) < N) ++L;
  c.level_off.assign(L + 2, 0);
  for (int l = 0; l <= L; ++l) {
    int64_t m = N >> l;
    c.level_off[l + 1] = c.level_off[l] + m * m * m;
  }
  c.mips.assign(c.level_off[L + 1], 0.0);
  for (int64_t v = 0; v < (int64_t)N * N * N; ++v)
    c.mips[v] = std::min(1.0, (double)c.occ_nom[v] / (double)c.Q);
  for (int l = 1; l <= L; ++l) {
    int64_t m = N >> l, mp = N >> (l - 1);
    double* dst = &c.mips[c.level_off[l]];
    const double* src = &c.mips[c.level_off[l - 1]];
    for (int64_t z = 0; z < m; ++z)
      for (int64_t y = 0; y < m; ++y)
        for (int64_t x = 0; x < m; ++x) {
          double s = 0;
          for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
              for (int dx = 0; dx < 2; ++dx)
                s += src[((2 * z + dz) * mp + (2 * y + dy)) * mp + (2 * x + dx)];
          dst[(z * m + y) * m + x] = s / 8.0;
        }
  }
  c.have_mips = true;
}

int n_levels(const Ctx& c) { return (int)c.level_off.size() - 1; }

double texel(const Ctx& c, int l, int64_t x, int64_t y, int64_t z) {
  int64_t m = c.N >> l;
  if (x < 0 || y < 0 || z < 0 || x >= m || y >= m || z >= m) return 0.0;
  return c.mips[c.level_off[l] + (z * m + y) * m + x];
}

double trilinear(const Ctx& c, int l, V3 q) {
  double s = (double)(1 << l);
  double u[3] = {q.x / s - 0.5, q.y / s - 0.5, q.z / s - 0.5};
  int64_t i0[3];
  double f[3];
  for (int k = 0; k < 3; ++k) { i0[k] = (int64_t)std::floor(u[k]); f[k] = u[k] - i0[k]; }
  double acc = 0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        double w = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) * (dz ? f[2] : 1 - f[2]);
        acc += w * texel(c, l, i0[0] + dx, i0[1] + dy, i0[2] + dz);
      }
  return acc;
}

// Cone-traced ambient occlusion at P: six cones along +-x, +-y, +-z whose half
// angle (cos = 2/3) makes them tile the sphere; each samples the pyramid at the
// level matching its diameter, front-to-back accumulated; no early exit.
double ambient_occlusion(const Ctx& c, V3 P) {
  const double tan_half = std::sqrt(5.0) / 2.0;
  const int maxl = n_levels(c) - 1;
  double sumA = 0;
  for (int cone = 0; cone < 6; ++cone) {
    V3 e = {0, 0, 0};
    double sg = (cone & 1) ? -1.0 : 1.0;
    if (cone / 2 == 0) e.x = sg; else if (cone / 2 == 1) e.y = sg; else e.z = sg;
    double A = 0, t = 1.0;
    while (t <= 16.0) {
      double dia = std::max(1.0, 2.0 * t * tan_half);
      double lam = std::log2(dia);
      if (lam > maxl) lam = maxl;
      int l0 = (int)std::floor(lam);
      double fl = lam - l0;
      V3 q = P + t * e;
      double s = trilinear(c, l0, q);
      if (fl > 0 && l0 + 1 <= maxl) s = (1 - fl) * s + fl * trilinear(c, l0 + 1, q);
      A = A + (1 - A) * s;
      t += dia / 2.0;
    }
    sumA += A;
  }
  return 1.0 - sumA / 6.0;
}

// Voxel-space shading (Sec. 3.4, Shading): at the centre P of voxel (x, y, z),
// ambient occlusion by the six cones above (when ao_cones is set) times a
// directional shadow term 1/2 + S/2. S is the transmittance of a ray from P
// toward the light through the base occupancy level: samples at P + k L for
// k = 1, 2, ... (one voxel apart, so the voxel's own lines do not shadow it),
// trilinear at texel centres, accumulated A <- A + (1 - A) s, S = 1 - A. The
// march ends where a sample's texels all lie outside the grid (beyond half a
// voxel past the boundary), so every sample that can be non-zero is taken.
double voxel_shade(const Ctx& c, int64_t x, int64_t y, int64_t z, const Params& prm) {
  const V3 P = {x + 0.5, y + 0.5, z + 0.5};
  const double ao = prm.ao_cones ? ambient_occlusion(c, P) : 1.0;
  const double lo = -0.5, hi = c.N + 0.5;
  double A = 0;
  for (int64_t k = 1;; ++k) {
    const V3 q = P + (double)k * prm.light;
    if (q.x < lo || q.x > hi || q.y < lo || q.y > hi || q.z < lo || q.z > hi) break;
    A = A + (1 - A) * trilinear(c, 0, q);
  }
  return ao * (0.5 + 0.5 * (1.0 - A));
}

// The shading field at a hit point: trilinear over the voxel-centre values,
// texel coordinates clamped to the grid (one texture sample per hit, Sec. 3.4).
double shade_at(const Ctx& c, V3 P, const Params& prm) {
  const double u[3] = {P.x - 0.5, P.y - 0.5, P.z - 0.5};
  int64_t i0[3];
  double f[3];
  for (int k = 0; k < 3; ++k) { i0[k] = (int64_t)std::floor(u[k]); f[k] = u[k] - i0[k]; }
  auto cl = [&](int64_t v) { return std::min<int64_t>(c.N - 1, std::max<int64_t>(0, v)); };
  double acc = 0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        double w = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) * (dz ? f[2] : 1 - f[2]);
        if (w == 0) continue;
        acc += w * voxel_shade(c, cl(i0[0] + dx), cl(i0[1] + dy), cl(i0[2] + dz), prm);
      }
  return acc;
}

// ------------------------------------------------------------------ rendering
struct Ray { V3 o, d; };

Ray camera_ray(const Camera& cam, int px, int py) {
  V3 eye = {cam.eye[0], cam.eye[1], cam.eye[2]};
  V3 tgt = {cam.target[0], cam.target[1], cam.target[2]};
  V3 up = {cam.up[0], cam.up[1], cam.up[2]};
  V3 f = normalize(tgt - eye);
  V3 rt = normalize(cross(f, up));
  V3 u = cross(rt, f);
  double W = cam.width, H = cam.height;
  Ray r;
  if (cam.ortho) {
    double oh = cam.ortho_h, ow = oh * W / H;
    r.o = eye + ((px + 0.5) / W - 0.5) * ow * rt + (0.5 - (py + 0.5) / H) * oh * u;
    r.d = f;
  } else {
    double th = std::tan(cam.fovy_deg * M_PI / 360.0);
    double sx = (2.0 * (px + 0.5) / W - 1.0) * th * (W / H);
    double sy = (1.0 - 2.0 * (py + 0.5) / H) * th;
    r.o = eye;
    r.d = normalize(f + sx * rt + sy * u);
  }
  return r;
}

// One candidate hit of a segment on a ray.
struct Cand {
  double t;
  uint32_t id;
  bool hit;        // accepted by the fp64 decisions
  bool fragile;    // a deciding predicate sits in its near-tie band
};

// Evaluate segment i against the ray. Returns true for an accepted hit, and for
// a rejected one (or a near miss) that a rounding of a deciding predicate could
// turn into a hit; `out.fragile` marks both kinds of near-tie.
bool eval_segment(const Ctx& c, const Ray& ray, uint32_t i, const Params& prm, Cand& out) {
  double nd;
  Hit h = line_capsule_entry(ray.o, ray.d, c.pos[i], c.pos[i + 1], c.r, &nd);
  bool graze = nd <= prm.graze_rel;
  if (!std::isfinite(h.t)) {
    if (!graze) return false;
    // near miss: its depth is the closest approach to the segment's midpoint
    out = {dot(0.5 * (c.pos[i] + c.pos[i + 1]) - ray.o, ray.d), i, false, true};
    return true;
  }
  const double t = h.t;
  const double band = prm.pos_abs + prm.pos_rel * std::fabs(t);
  bool fragile = graze || std::fabs(t) <= band;
  bool ok = t >= 0;
  V3 P = ray.o + t * ray.d;
  for (int k = 0; k < 3; ++k) {
    double pk = comp(P, k);
    if (pk < 0 || pk > c.N) ok = false;
    if (std::fabs(pk) <= band || std::fabs(pk - c.N) <= band) fragile = true;
  }
  if (c.en[i]) {
    double s = dot(P - c.pos[i], c.nrm[i]);
    if (s < 0) ok = false;
    if (std::fabs(s) <= band) fragile = true;
  }
  if (c.en[i + 1]) {
    double s = dot(P - c.pos[i + 1], c.nrm[i + 1]);
    if (s > 0) ok = false;
    if (std::fabs(s) <= band) fragile = true;
  }
  if (!ok && !fragile) return false;
  out = {t, i, ok, fragile};
  return true;
}

// Tangent colouring: |unit direction| per component.
V3 seg_colour(const Ctx& c, uint32_t i) {
  V3 d = c.pos[i + 1] - c.pos[i];
  double n = norm(d);
  if (n == 0) return {1, 1, 1};
  return {std::fabs(d.x) / n, std::fabs(d.y) / n, std::fabs(d.z) / n};
}

struct PixelOut {
  float rgba[4], rgba_alt[4];
  int32_t id, id_alt;
  float t;
  uint8_t exempt;  // bit0: colour exempt; bit1: first-id exempt
};

// Front-to-back compositing of the accepted hits in (t, id) order over
// transparent black: premultiplied colour C += T * alpha * c * shade (shade =
// AO per hit, the voxel-space shading field, or 1), transmittance
// T *= 1 - alpha; output (C, 1 - T).
void composite(const Ctx& c, const Ray& ray, const std::vector<Cand>& cs, int toggle,
               const Params& prm, double out[4]) {
  double C[3] = {0, 0, 0}, T = 1.0;
  for (size_t k = 0; k < cs.size(); ++k) {
    bool use = ((int)k == toggle) ? !cs[k].hit : cs[k].hit;
    if (!use) continue;
    if (T < 1e-12) break;
    V3 col = seg_colour(c, cs[k].id);
    if (prm.voxel_shading) col = shade_at(c, ray.o + cs[k].t * ray.d, prm) * col;
    else if (prm.ao_cones) col = ambient_occlusion(c, ray.o + cs[k].t * ray.d) * col;
    C[0] += T * prm.alpha * col.x;
    C[1] += T * prm.alpha * col.y;
    C[2] += T * prm.alpha * col.z;
    T *= (1.0 - prm.alpha);
  }
  out[0] = C[0]; out[1] = C[1]; out[2] = C[2]; out[3] = 1.0 - T;
}

int first_hit(const std::vector<Cand>& cs, int toggle) {
  for (size_t k = 0; k < cs.size(); ++k) {
    bool use = ((int)k == toggle) ? !cs[k].hit : cs[k].hit;
    if (use) return (int)k;
  }
  return -1;
}

// Resolve one pixel: the primary result from the fp64 decisions, plus one
// alternative when exactly one near-tie event (a fragile candidate flipping, or
// two tied hits swapping) could change it; more than one event exempts it.
void resolve_pixel(const Ctx& c, const Ray& ray, std::vector<Cand>& cs, const Params& prm,
                   PixelOut& po) {
  std::sort(cs.begin(), cs.end(), [](const Cand& a, const Cand& b) {
    return a.t < b.t || (a.t == b.t && a.id < b.id);
  });
  auto tieband = [&](double t) { return prm.tie_abs + prm.tie_rel * std::fabs(t); };
  double rgba[4];
  composite(c, ray, cs, -1, prm, rgba);
  int f = first_hit(cs, -1);
  po.id = f < 0 ? -1 : (int32_t)cs[f].id;
  po.t = f < 0 ? INFINITY : (float)cs[f].t;
  po.id_alt = po.id;
  for (int k = 0; k < 4; ++k) po.rgba[k] = po.rgba_alt[k] = (float)rgba[k];
  po.exempt = 0;

  // horizon: past it, transmittance of the primary sequence is below T_STOP / 10
  double horizon = INFINITY;
  {
    double T = 1.0;
    for (const Cand& h : cs) {
      if (!h.hit) continue;
      T *= 1.0 - prm.alpha;
      if (T < T_STOP * 0.1) { horizon = h.t; break; }
    }
  }
  // accepted hits in order, for ties
  std::vector<int> acc;
  for (size_t k = 0; k < cs.size(); ++k)
    if (cs[k].hit) acc.push_back((int)k);

  // ---- first id
  {
    double tf = f < 0 ? horizon : cs[f].t;
    std::vector<int> ev;  // fragile candidates at or before the first hit
    for (size_t k = 0; k < cs.size(); ++k) {
      if (cs[k].t > tf + tieband(tf)) break;
      if (cs[k].fragile) ev.push_back((int)k);
    }
    bool tie01 = acc.size() > 1 && std::fabs(cs[acc[1]].t - cs[acc[0]].t) <= tieband(cs[acc[1]].t);
    int n_ev = (int)ev.size() + (tie01 ? 1 : 0);
    if (n_ev == 1) {
      if (tie01) {
        po.id_alt = (int32_t)cs[acc[1]].id;
      } else {
        int g = first_hit(cs, ev[0]);
        po.id_alt = g < 0 ? -1 : (int32_t)cs[g].id;
      }
    } else if (n_ev > 1) {
      po.exempt |= 2;
    }
  }

  // ---- colour
  {
    std::vector<int> ev;
    for (size_t k = 0; k < cs.size(); ++k) {
      if (cs[k].t > horizon + tieband(horizon)) break;
      if (cs[k].fragile) ev.push_back((int)k);
    }
    std::vector<int> ties;  // index into acc: acc[j] and acc[j+1] swap
    for (size_t j = 0; j + 1 < acc.size(); ++j) {
      double ta = cs[acc[j]].t, tb = cs[acc[j + 1]].t;
      if (ta > horizon + tieband(horizon)) break;
      if (std::fabs(tb - ta) > tieband(tb)) continue;
      std::vector<Cand> sw = cs;
      std::swap(sw[acc[j]], sw[acc[j + 1]]);
      double alt[4];
      composite(c, ray, sw, -1, prm, alt);
      double dmax = 0;
      for (int q = 0; q < 4; ++q) dmax = std::max(dmax, std::fabs(alt[q] - rgba[q]));
      if (dmax > 1e-4) ties.push_back((int)j);
    }
    size_t n_ev = ev.size() + ties.size();
    if (n_ev == 1) {
      double alt[4];
      if (!ties.empty()) {
        std::vector<Cand> sw = cs;
        std::swap(sw[acc[ties[0]]], sw[acc[ties[0] + 1]]);
        composite(c, ray, sw, -1, prm, alt);
      } else {
        composite(c, ray, cs, ev[0], prm, alt);
      }
      for (int q = 0; q < 4; ++q) po.rgba_alt[q] = (float)alt[q];
    } else if (n_ev > 1) {
      po.exempt |= 1;
    }
  }
}

// Ray against the grid box [0, N]^3: entry/exit parameters (t >= 0 only).
bool box_clip(const Ray& ray, double N, double& t0, double& t1) {
  t0 = 0; t1 = INFINITY;
  for (int k = 0; k < 3; ++k) {
    double o = comp(ray.o, k), d = comp(ray.d, k);
    if (d == 0) {
      if (o < 0 || o > N) return false;
      continue;
    }
    double a = (0 - o) / d, b = (N - o) / d;
    if (a > b) std::swap(a, b);
    t0 = std::max(t0, a);
    t1 = std::min(t1, b);
  }
  return t0 <= t1;
}

void render_pixel(const Ctx& c, const Camera& cam, const Params& prm, int px, int py, bool brute,
                  PixelOut& po) {
  Ray ray = camera_ray(cam, px, py);
  std::vector<Cand> cs;
  if (brute) {
    for (int64_t i = 0; i < c.V; ++i) {
      if (!seg_valid(c, i)) continue;
      Cand cd;
      if (eval_segment(c, ray, (uint32_t)i, prm, cd)) cs.push_back(cd);
    }
    resolve_pixel(c, ray, cs, prm, po);
    return;
  }
  // Walk the voxels the ray crosses (Amanatides & Woo), gathering every listed
  // segment once. A hit point lies in a voxel of the walk and that voxel lists
  // the segment, so after the voxel whose exit is t_x every hit before t_x is
  // known.
  double t0, t1;
  std::unordered_set<uint32_t> seen;
  if (box_clip(ray, c.N, t0, t1)) {
    const int N = c.N;
    V3 p = ray.o + t0 * ray.d;
    int64_t v[3], step[3];
    double tnext[3], tdelta[3];
    for (int k = 0; k < 3; ++k) {
      double pk = comp(p, k), dk = comp(ray.d, k);
      v[k] = std::min<int64_t>(N - 1, std::max<int64_t>(0, (int64_t)std::floor(pk)));
      if (dk > 0) { step[k] = 1; tnext[k] = ((v[k] + 1) - comp(ray.o, k)) / dk; tdelta[k] = 1 / dk; }
      else if (dk < 0) { step[k] = -1; tnext[k] = (v[k] - comp(ray.o, k)) / dk; tdelta[k] = -1 / dk; }
      else { step[k] = 0; tnext[k] = INFINITY; tdelta[k] = INFINITY; }
    }
    for (;;) {
      int64_t vi = (v[2] * N + v[1]) * N + v[0];
      for (uint64_t s = c.start[vi]; s < c.start[vi + 1]; ++s) {
        uint32_t id = c.ids[s];
        if (!seen.insert(id).second) continue;
        Cand cd;
        if (eval_segment(c, ray, id, prm, cd)) cs.push_back(cd);
      }
      int k = 0;
      if (tnext[1] < tnext[k]) k = 1;
      if (tnext[2] < tnext[k]) k = 2;
      double texit = tnext[k];
      // stop once the accepted hits safely before texit already take the
      // transmittance past the horizon used by resolve_pixel
      double safe = texit - 2 * (prm.tie_abs + prm.tie_rel * std::fabs(texit)) - 1e-3;
      int n_before = 0;
      for (const Cand& cd : cs)
        if (cd.hit && cd.t < safe) n_before++;
      if (n_before > 0 && std::pow(1.0 - prm.alpha, n_before) < T_STOP * 1e-2) break;
      if (texit > t1) break;
      v[k] += step[k];
      tnext[k] += tdelta[k];
      if (v[k] < 0 || v[k] >= N) break;
    }
  }
  resolve_pixel(c, ray, cs, prm, po);
}

}  // namespace

// ============================================================== C interface
extern "C" {

struct or_camera {
  int32_t width, height, ortho;
  float eye[3], target[3], up[3], fovy_deg, ortho_h;
};
struct or_params {
  float alpha;
  int32_t ao_cones;
  double tie_rel, tie_abs, graze_rel, pos_abs, pos_rel;
  int32_t voxel_shading;
  float light[3];  // direction toward the light (normalized here)
};

Params make_params(const or_params* p) {
  Params prm;
  prm.alpha = p->alpha; prm.ao_cones = p->ao_cones;
  prm.tie_rel = p->tie_rel; prm.tie_abs = p->tie_abs;
  prm.graze_rel = p->graze_rel;
  prm.pos_abs = p->pos_abs; prm.pos_rel = p->pos_rel;
  prm.voxel_shading = p->voxel_shading;
  const V3 l = {p->light[0], p->light[1], p->light[2]};
  prm.light = norm(l) > 0 ? normalize(l) : V3{0, 0, 1};
  return prm;
}

void need_mips(Ctx* c) {
  if (!c->have_mips) { if (!c->have_lists) build_lists(*c); build_mips(*c); }
}

// Returns 0 on success; 1 = bad grid side; 2 = coordinate out of range or not
// finite; 3 = bad offsets; 4 = bad radius.
void* or_create(const float* xyz, int32_t stride, int64_t V, const int64_t* offsets, int64_t P,
                int32_t N, float radius, float r_min, int32_t occ_scale, int32_t nthreads,
                int32_t* status) {
  Ctx* c = new Ctx();
  *status = 0;
  c->N = N; c->V = V; c->P = P; c->nthreads = nthreads > 0 ? nthreads : 1;
  c->Q = occ_scale > 0 ? occ_scale : 32;
  c->r_min = r_min;
  if (N < 16 || N > 512 || (N & (N - 1))) { *status = 1; return c; }
  if (!(radius > 0) || radius > 4.0f) { *status = 4; return c; }
  c->R = (int64_t)std::nearbyint((double)radius * UNITS);
  c->RL = c->R + LIST_MARGIN_UNITS;
  c->r = (double)c->R / UNITS;
  c->X.resize(3 * V);
  c->pos.resize(V);
  for (int64_t i = 0; i < V; ++i) {
    for (int k = 0; k < 3; ++k) {
      double x = xyz[i * stride + k];
      if (!std::isfinite(x) || x < -256.0 || x >= 768.0) { *status = 2; return c; }
      c->X[3 * i + k] = (int64_t)std::nearbyint(x * (double)UNITS);
    }
    c->pos[i] = {c->X[3 * i] / (double)UNITS, c->X[3 * i + 1] / (double)UNITS,
                 c->X[3 * i + 2] / (double)UNITS};
  }
  c->first.assign(V, 0); c->last.assign(V, 0);
  if (offsets[0] != 0 || offsets[P] != V) { *status = 3; return c; }
  for (int64_t p = 0; p < P; ++p) {
    if (offsets[p + 1] < offsets[p]) { *status = 3; return c; }
    if (offsets[p + 1] > offsets[p]) {
      c->first[offsets[p]] = 1;
      c->last[offsets[p + 1] - 1] = 1;
    }
  }
  // clip normals: central-difference tangent at interior vertices
  c->nrm.assign(V, {0, 0, 0});
  c->en.assign(V, 0);
  for (int64_t i = 0; i < V; ++i) {
    if (c->first[i] || c->last[i]) continue;
    V3 t = c->pos[i + 1] - c->pos[i - 1];
    double n = norm(t);
    if (n > 0) { c->nrm[i] = (1.0 / n) * t; c->en[i] = 1; }
  }
  return c;
}

void or_destroy(void* h) { delete (Ctx*)h; }

int64_t or_build_lists(void* h) {
  Ctx* c = (Ctx*)h;
  build_lists(*c);
  return (int64_t)c->ids.size();
}

int64_t or_ambiguous(void* h) { return ((Ctx*)h)->F_ambiguous; }

void or_get_lists(void* h, uint32_t* count, uint32_t* occ_nom, uint32_t* occ_lo,
                  uint32_t* occ_hi, uint64_t* start, uint32_t* ids) {
  Ctx* c = (Ctx*)h;
  int64_t nv = (int64_t)c->N * c->N * c->N;
  for (int64_t v = 0; v < nv; ++v) {
    if (count) count[v] = (uint32_t)(c->start[v + 1] - c->start[v]);
    if (occ_nom) occ_nom[v] = c->occ_nom[v];
    if (occ_lo) occ_lo[v] = c->occ_lo[v];
    if (occ_hi) occ_hi[v] = c->occ_hi[v];
  }
  if (start) std::memcpy(start, c->start.data(), sizeof(uint64_t) * (nv + 1));
  if (ids) std::memcpy(ids, c->ids.data(), sizeof(uint32_t) * c->ids.size());
}

void or_get_vertices(void* h, double* pos, double* nrm, uint8_t* en, uint8_t* first,
                     uint8_t* last) {
  Ctx* c = (Ctx*)h;
  for (int64_t i = 0; i < c->V; ++i) {
    if (pos) { pos[3 * i] = c->pos[i].x; pos[3 * i + 1] = c->pos[i].y; pos[3 * i + 2] = c->pos[i].z; }
    if (nrm) { nrm[3 * i] = c->nrm[i].x; nrm[3 * i + 1] = c->nrm[i].y; nrm[3 * i + 2] = c->nrm[i].z; }
    if (en) en[i] = c->en[i];
    if (first) first[i] = c->first[i];
    if (last) last[i] = c->last[i];
  }
}

int64_t or_build_mips(void* h, double* out) {
  Ctx* c = (Ctx*)h;
  if (!c->have_lists) build_lists(*c);
  build_mips(*c);
  if (out) std::memcpy(out, c->mips.data(), sizeof(double) * c->mips.size());
  return (int64_t)c->mips.size();
}

// Voxel-space shading value at the centre of voxel (x, y, z).
double or_voxel_shade(void* h, int64_t x, int64_t y, int64_t z, int32_t ao_cones,
                      const float* light) {
  Ctx* c = (Ctx*)h;
  need_mips(c);
  or_params p;
  std::memset(&p, 0, sizeof(p));
  p.ao_cones = ao_cones;
  p.voxel_shading = 1;
  for (int k = 0; k < 3; ++k) p.light[k] = light[k];
  return voxel_shade(*c, x, y, z, make_params(&p));
}

double or_ao(void* h, const double* P) {
  Ctx* c = (Ctx*)h;
  if (!c->have_mips) { if (!c->have_lists) build_lists(*c); build_mips(*c); }
  return ambient_occlusion(*c, V3{P[0], P[1], P[2]});
}

// Render pixels [pix_begin, pix_end) (row-major, row 0 at the top). Outputs are
// indexed relative to pix_begin. brute != 0 ignores the lists.
int32_t or_render(void* h, const or_camera* cam_in, const or_params* prm_in, int32_t brute,
                  int64_t pix_begin, int64_t pix_end, float* rgba, float* rgba_alt,
                  int32_t* first_id, int32_t* first_id_alt, float* first_t, uint8_t* exempt) {
  Ctx* c = (Ctx*)h;
  if (!brute && !c->have_lists) build_lists(*c);
  if (prm_in->ao_cones || prm_in->voxel_shading) need_mips(c);
  Camera cam;
  cam.width = cam_in->width; cam.height = cam_in->height; cam.ortho = cam_in->ortho;
  for (int k = 0; k < 3; ++k) {
    cam.eye[k] = cam_in->eye[k]; cam.target[k] = cam_in->target[k]; cam.up[k] = cam_in->up[k];
  }
  cam.fovy_deg = cam_in->fovy_deg; cam.ortho_h = cam_in->ortho_h;
  const Params prm = make_params(prm_in);
  int64_t n = pix_end - pix_begin;
  parallel_for(n, c->nthreads, [&](int64_t j) {
    int64_t p = pix_begin + j;
    int px = (int)(p % cam.width), py = (int)(p / cam.width);
    PixelOut po;
    render_pixel(*c, cam, prm, px, py, brute != 0, po);
    for (int k = 0; k < 4; ++k) {
      if (rgba) rgba[4 * j + k] = po.rgba[k];
      if (rgba_alt) rgba_alt[4 * j + k] = po.rgba_alt[k];
    }
    if (first_id) first_id[j] = po.id;
    if (first_id_alt) first_id_alt[j] = po.id_alt;
    if (first_t) first_t[j] = po.t;
    if (exempt) exempt[j] = po.exempt;
  });
  return 0;
}

// Fragments of one voxel by brute force over every segment (no list build): the
// same exact predicate and codes as the list build, for sampled checks of sets
// too large for a full build. Returns the count; writes up to `cap` ids in
// increasing order and occ[0..2] = nominal, lowest and highest code sums.
int64_t or_voxel_fragments(void* h, int64_t x, int64_t y, int64_t z, uint32_t* ids, int64_t cap,
                           uint64_t* occ) {
  Ctx* c = (Ctx*)h;
  const int64_t n_chunks = 256;
  const int64_t per = (c->V + n_chunks - 1) / n_chunks;
  std::vector<std::vector<uint32_t>> found(n_chunks);
  std::vector<uint64_t> on(n_chunks, 0), ol(n_chunks, 0), oh(n_chunks, 0);
  parallel_for(n_chunks, c->nthreads, [&](int64_t k) {
    for (int64_t i = k * per; i < std::min(c->V, (k + 1) * per); ++i) {
      if (!seg_valid(*c, i)) continue;
      int64_t vlo[3], vhi[3];
      seg_voxel_range(*c, i, vlo, vhi);
      if (x < vlo[0] || x > vhi[0] || y < vlo[1] || y > vhi[1] || z < vlo[2] || z > vhi[2]) continue;
      uint32_t qn, ql, qh;
      bool a;
      if (!fragment(*c, i, x, y, z, qn, ql, qh, a)) continue;
      found[k].push_back((uint32_t)i);
      on[k] += qn; ol[k] += ql; oh[k] += qh;
    }
  }, 1);
  int64_t n = 0;
  uint64_t s0 = 0, s1 = 0, s2 = 0;
  for (int64_t k = 0; k < n_chunks; ++k) {
    for (uint32_t id : found[k]) {
      if (ids && n < cap) ids[n] = id;
      ++n;
    }
    s0 += on[k]; s1 += ol[k]; s2 += oh[k];
  }
  if (occ) { occ[0] = s0; occ[1] = s1; occ[2] = s2; }
  return n;
}

// Render the n pixels listed in pix (row-major indices), one per thread, into
// outputs indexed like pix.
int32_t or_render_pixels(void* h, const or_camera* cam_in, const or_params* prm_in, int32_t brute,
                         const int64_t* pix, int64_t n, float* rgba, float* rgba_alt,
                         int32_t* first_id, int32_t* first_id_alt, float* first_t, uint8_t* exempt) {
  Ctx* c = (Ctx*)h;
  if (!brute && !c->have_lists) build_lists(*c);
  if (prm_in->ao_cones || prm_in->voxel_shading) need_mips(c);
  Camera cam;
  cam.width = cam_in->width; cam.height = cam_in->height; cam.ortho = cam_in->ortho;
  for (int k = 0; k < 3; ++k) {
    cam.eye[k] = cam_in->eye[k]; cam.target[k] = cam_in->target[k]; cam.up[k] = cam_in->up[k];
  }
  cam.fovy_deg = cam_in->fovy_deg; cam.ortho_h = cam_in->ortho_h;
  const Params prm = make_params(prm_in);
  parallel_for(n, c->nthreads, [&](int64_t j) {
    const int64_t p = pix[j];
    int px = (int)(p % cam.width), py = (int)(p / cam.width);
    PixelOut po;
    render_pixel(*c, cam, prm, px, py, brute != 0, po);
    for (int k = 0; k < 4; ++k) {
      if (rgba) rgba[4 * j + k] = po.rgba[k];
      if (rgba_alt) rgba_alt[4 * j + k] = po.rgba_alt[k];
    }
    if (first_id) first_id[j] = po.id;
    if (first_id_alt) first_id_alt[j] = po.id_alt;
    if (first_t) first_t[j] = po.t;
    if (exempt) exempt[j] = po.exempt;
  }, 1);
  return 0;
}

// ----- single-function entry points for pins
int32_t or_seg_box_within(const int64_t* A, const int64_t* B, const int64_t* lo, int64_t S,
                          int64_t R) {
  return seg_box_within(A, B, lo, S, R) ? 1 : 0;
}

double or_clipped_capsule_sdf(const double* p, const double* v0, const double* v1,
                              const double* n0, const double* n1, int32_t en0, int32_t en1,
                              double r) {
  return clipped_capsule_sdf({p[0], p[1], p[2]}, {v0[0], v0[1], v0[2]}, {v1[0], v1[1], v1[2]},
                             {n0[0], n0[1], n0[2]}, {n1[0], n1[1], n1[2]}, en0, en1, r);
}

double or_capsule_occupancy(const double* p, const double* v0, const double* v1,
                            const double* n0, const double* n1, int32_t en0, int32_t en1,
                            double r, double r_min) {
  return capsule_occupancy({p[0], p[1], p[2]}, {v0[0], v0[1], v0[2]}, {v1[0], v1[1], v1[2]},
                           {n0[0], n0[1], n0[2]}, {n1[0], n1[1], n1[2]}, en0, en1, r, r_min);
}

// First entry parameter of the line o + t d (d normalised here) into the capsule;
// +inf when the line misses.
double or_line_capsule_entry(const double* o, const double* d, const double* a, const double* b,
                             double r) {
  V3 dd = normalize(V3{d[0], d[1], d[2]});
  Hit h = line_capsule_entry({o[0], o[1], o[2]}, dd, {a[0], a[1], a[2]}, {b[0], b[1], b[2]}, r,
                             nullptr);
  return h.t;
}

void or_camera_ray(const or_camera* cam_in, int32_t px, int32_t py, double* o, double* d) {
  Camera cam;
  cam.width = cam_in->width; cam.height = cam_in->height; cam.ortho = cam_in->ortho;
  for (int k = 0; k < 3; ++k) {
    cam.eye[k] = cam_in->eye[k]; cam.target[k] = cam_in->target[k]; cam.up[k] = cam_in->up[k];
  }
  cam.fovy_deg = cam_in->fovy_deg; cam.ortho_h = cam_in->ortho_h;
  Ray r = camera_ray(cam, px, py);
  o[0] = r.o.x; o[1] = r.o.y; o[2] = r.o.z;
  d[0] = r.d.x; d[1] = r.d.y; d[2] = r.d.z;
}

}  // extern "C"
