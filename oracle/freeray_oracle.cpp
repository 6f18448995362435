// Plain, slow FP64 CPU oracle for the differentiable freeform-lens trace of
// de Koning, Heemels, Adam and Moeller, "Gradient descent-based freeform optics
// design using algorithmic differentiable non-sequential ray tracing" (2023).
//
// TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
// CPU-baseline / reference leg load this library. The product (CUDA) path never
// does, and this file shares no code, header, table or constant with it.
//
// What it computes, in the paper's order and notation:
//   Sec. 2.1   clamped uniform knot vector (Eq. knot vector + equispaced interior
//              knots), Cox-de Boor basis (Eq. Cox-de Boor, second denominator read
//              as u_{i+p+1}-u_{i+1}), tensor-product surface (Eq. Bsplinesurfacedef),
//              linear X,Y through the Greville construction (Eqs. linearX/linearY)
//              and their inverses.
//   Sec. 2.2.1 sources: collimated rays on a square grid of [0,1]^2 with d=(0,0,1);
//              point source with theta ~ U[0,2pi), phi = arccos(1-(1-cos phi_max) a).
//              The random numbers come from Philox-4x32-10 (Salmon et al., SC'11),
//              written here from its published definition.
//   Sec. 2.2.1 ray/freeform intersection: the smallest positive root of
//              f(t) = Z(o_uv + d_uv t) - d_z t - o_z (Eq. surfaceintersect), found
//              by a uniform scan of the convex-hull bracket followed by bisection to
//              FP64 precision. This is the definition, not the paper's triangle mesh.
//   Sec. 2.2   refraction at the flat entry face and at the freeform (vector Snell
//              law), total internal reflection culled, Schlick transmission weights.
//   Sec. 2.3   screen pixels, ghost pixels, Gaussian reconstruction filter
//              (Eq. filter1dim) normalised over all pixels, irradiance sum
//              I_ij = sum_k w_k F_ij(x_k), divided by the pixel area.
//   Loss       squared L2 over the interior pixels, and its gradient dL/dE;
//              the paper's loss (Sec. 2.5, Eq. pipelineLoss): the Frobenius norm of
//              the difference of the sum-normalised images over sqrt(nx ny), and its
//              gradient through both normalisations.
//   Reparam.   control heights from unconstrained variables through tanh and the
//              affine map onto (z_min, z_max), plus an offset f(P^x, P^y) taken at
//              the Greville points (Sec. 2.4.2, Eqs. outputcorrection and
//              outputcorrectionwfunc; spherical offsets of Table magndata).
//   Gradient   dL/dP^z by forward-mode dual numbers carried through this same
//              trace (an exact derivative of the code above), with the implicit
//              function theorem at the FP64 root for the point source.
//   Adam       Kingma & Ba, Algorithm 1.
//
// Every function is pinned by tests/test_oracle_*.py (closed forms, library
// routines, invariants, finite differences); no part is "parity unpinned".

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <type_traits>
#include <vector>

extern "C" {

// ----------------------------------------------------------------------------
// Public structures of the oracle (its own; not shared with the CUDA library).
// ----------------------------------------------------------------------------
typedef struct or_problem {
  // Lens (Sec. 2.1): control net (n1+1) x (n2+1), degrees (p,q), heights P^z
  // row-major with the u index i slow: P[i*(n2+1)+j].
  int32_t n1, n2, p, q;
  const double* P;
  double rx, ry;      // lens half-widths r_x, r_y
  double z_in;        // flat entry face z = z_in
  double n_glass;     // refractive index of the lens (outside: air, 1)
  // Source (Sec. 2.2.1).
  int32_t src_kind;   // 0 collimated, 1 point source(s)
  int32_t cols, rows; // collimated: ray grid cols x rows over [0,1]^2
  int32_t jitter;     // collimated: 0 cell centres, 1 Philox jitter in the cell
  double src_pos[3];  // point: centre of the source (grid)
  double half_angle;  // point: phi_max in radians
  int32_t grid_nx, grid_ny;  // point: grid of point sources (1,1 = single)
  double grid_w, grid_h;     // point: extent of the grid of sources
  double flux;        // total flux Phi of the source, split evenly over rays
  uint64_t n_rays;    // total number of rays of the source
  uint64_t seed;      // Philox key
  // Target (Sec. 2.3).
  double z_screen, Rx, Ry;   // screen plane and its half-widths
  int32_t nx, ny;            // interior pixels
  int32_t nu_x, nu_y;        // filter sizes (odd); ghost pixels (nu-1)/2 per side
  double alpha;              // Gaussian filter coefficient, in pixel units
  int32_t scan_points;       // root scan resolution (>= 16)
  // Point-source intersection (Sec. 2.2.2): 0 = the B-spline itself (smallest
  // positive root of Eq. surfaceintersect); > 0 = the triangle mesh that splits
  // every knot span product into mesh_nu x mesh_nv rectangles, two triangles each.
  int32_t mesh_nu;
  int32_t mesh_nv;
  int32_t pad_;
  // Optional freeform entry face (both faces optimised, Sec. 4): heights
  // P_in (n1_in+1) x (n2_in+1) of a second B-spline height field of degrees
  // (p,q) over the same aperture; NULL = the flat entry face z = z_in.
  const double* P_in;
  int32_t n1_in, n2_in;
} or_problem;

typedef struct or_record {
  int32_t status;            // OR_* below
  int32_t span_i, span_j;    // knot span of the freeform hit (index of u_i0, v_j0)
  int32_t pad_;
  double u, v;               // freeform hit in parameter space
  double x, y, z;            // freeform hit in space
  double dx, dy, dz;         // ray direction inside the glass
  double tx, ty, tz;         // ray direction after the freeform
  double X, Y;               // screen hit
  double w;                  // final ray weight
  double t;                  // intersection parameter inside the glass (point)
} or_record;

typedef struct or_stats {
  uint64_t counts[8];        // indexed by status
} or_stats;

}  // extern "C"

enum {
  OR_OK = 0,
  OR_APERTURE_MISS = 1,
  OR_OUT_OF_DOMAIN = 2,
  OR_TIR = 3,
  OR_OFF_SCREEN = 4,
  OR_INVALID = 5,
};

namespace {

// ----------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies, the key bumped by
// the Weyl constants between rounds.
// ----------------------------------------------------------------------------
void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    const uint64_t prod0 = M0 * c0;
    const uint64_t prod1 = M1 * c2;
    const uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    const uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// A 32-bit word to a uniform number in the open interval (0,1): the top 23
// bits plus one half, times 2^-23 (a value FP32 also holds exactly).
double word_to_unit(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }

// The two uniforms of ray `id`: counter (id_lo, id_hi, 0, 0), key = seed.
void ray_uniforms(uint64_t seed, uint64_t id, double* xi1, double* xi2) {
  const uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), 0u, 0u};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  philox4x32_10(ctr, key, out);
  *xi1 = word_to_unit(out[0]);
  *xi2 = word_to_unit(out[1]);
}

// ----------------------------------------------------------------------------
// Forward-mode dual numbers: a value and its derivatives along NT directions.
// ----------------------------------------------------------------------------
template <int NT>
struct Dual {
  double v;
  double d[NT];
  Dual() : v(0.0) { std::memset(d, 0, sizeof d); }
  Dual(double x) : v(x) { std::memset(d, 0, sizeof d); }  // NOLINT: implicit on purpose
};

template <int NT> Dual<NT> operator+(const Dual<NT>& a, const Dual<NT>& b) {
  Dual<NT> r; r.v = a.v + b.v; for (int k = 0; k < NT; ++k) r.d[k] = a.d[k] + b.d[k]; return r;
}
template <int NT> Dual<NT> operator-(const Dual<NT>& a, const Dual<NT>& b) {
  Dual<NT> r; r.v = a.v - b.v; for (int k = 0; k < NT; ++k) r.d[k] = a.d[k] - b.d[k]; return r;
}
template <int NT> Dual<NT> operator-(const Dual<NT>& a) {
  Dual<NT> r; r.v = -a.v; for (int k = 0; k < NT; ++k) r.d[k] = -a.d[k]; return r;
}
template <int NT> Dual<NT> operator*(const Dual<NT>& a, const Dual<NT>& b) {
  Dual<NT> r; r.v = a.v * b.v; for (int k = 0; k < NT; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r;
}
template <int NT> Dual<NT> operator/(const Dual<NT>& a, const Dual<NT>& b) {
  Dual<NT> r; r.v = a.v / b.v;
  for (int k = 0; k < NT; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) / b.v;
  return r;
}
template <int NT> Dual<NT> operator+(const Dual<NT>& a, double b) { return a + Dual<NT>(b); }
template <int NT> Dual<NT> operator+(double a, const Dual<NT>& b) { return Dual<NT>(a) + b; }
template <int NT> Dual<NT> operator-(const Dual<NT>& a, double b) { return a - Dual<NT>(b); }
template <int NT> Dual<NT> operator-(double a, const Dual<NT>& b) { return Dual<NT>(a) - b; }
template <int NT> Dual<NT> operator*(const Dual<NT>& a, double b) {
  Dual<NT> r; r.v = a.v * b; for (int k = 0; k < NT; ++k) r.d[k] = a.d[k] * b; return r;
}
template <int NT> Dual<NT> operator*(double a, const Dual<NT>& b) { return b * a; }
template <int NT> Dual<NT> operator/(const Dual<NT>& a, double b) { return a * (1.0 / b); }
template <int NT> Dual<NT> operator/(double a, const Dual<NT>& b) { return Dual<NT>(a) / b; }

template <int NT> Dual<NT> sqrt(const Dual<NT>& a) {
  Dual<NT> r; r.v = std::sqrt(a.v);
  for (int k = 0; k < NT; ++k) r.d[k] = a.d[k] / (2.0 * r.v);
  return r;
}
template <int NT> Dual<NT> exp(const Dual<NT>& a) {
  Dual<NT> r; r.v = std::exp(a.v);
  for (int k = 0; k < NT; ++k) r.d[k] = a.d[k] * r.v;
  return r;
}
template <int NT> Dual<NT> cos(const Dual<NT>& a) {
  Dual<NT> r; r.v = std::cos(a.v); const double s = -std::sin(a.v);
  for (int k = 0; k < NT; ++k) r.d[k] = a.d[k] * s;
  return r;
}
template <int NT> Dual<NT> sin(const Dual<NT>& a) {
  Dual<NT> r; r.v = std::sin(a.v); const double c = std::cos(a.v);
  for (int k = 0; k < NT; ++k) r.d[k] = a.d[k] * c;
  return r;
}

inline double val(double x) { return x; }
template <int NT> double val(const Dual<NT>& x) { return x.v; }
inline void seed_dir(double&, int) {}
template <int NT> void seed_dir(Dual<NT>& x, int k) { x.d[k] = 1.0; }
using std::sqrt;
using std::exp;
using std::cos;
using std::sin;

template <class T> T sq(const T& a) { return a * a; }

// ----------------------------------------------------------------------------
// Sec. 2.1: B-spline basis.
// ----------------------------------------------------------------------------

// Clamped knot vector with p+1 zeros, p+1 ones and equispaced interior knots
// u_i = (i-p)/(n-p+1), i = p..n+1. It has n+p+2 entries.
std::vector<double> clamped_uniform_knots(int n, int p) {
  std::vector<double> U(n + p + 2);
  for (int i = 0; i <= p; ++i) U[i] = 0.0;
  for (int i = p; i <= n + 1; ++i) U[i] = (double)(i - p) / (double)(n - p + 1);
  for (int i = n + 1; i <= n + p + 1; ++i) U[i] = 1.0;
  return U;
}

// N_{i,k}(u) by the Cox-de Boor recursion (Piegl & Tiller eq. 2.5), with 0/0 := 0.
// N_{i,0} is the indicator of the half-open span [u_i, u_{i+1}); at the right end
// u = u_last the last non-empty span is taken as closed, so that the clamped end
// value N_{n,p}(1) = 1 holds.
template <class T>
T basis(const std::vector<double>& U, int i, int k, const T& u) {
  const int m = (int)U.size() - 1;
  if (k == 0) {
    const double uv = val(u);
    bool inside = (U[i] <= uv && uv < U[i + 1]);
    if (!inside && uv == U[m] && U[i] < U[i + 1] && U[i + 1] == U[m]) inside = true;
    return T(inside ? 1.0 : 0.0);
  }
  T left(0.0), right(0.0);
  const double d1 = U[i + k] - U[i];
  const double d2 = U[i + k + 1] - U[i + 1];
  if (d1 != 0.0) left = (u - U[i]) / d1 * basis(U, i, k - 1, u);
  if (d2 != 0.0) right = (U[i + k + 1] - u) / d2 * basis(U, i + 1, k - 1, u);
  return left + right;
}

// dN_{i,k}/du = k/(u_{i+k}-u_i) N_{i,k-1} - k/(u_{i+k+1}-u_{i+1}) N_{i+1,k-1}
// (Piegl & Tiller eq. 2.7), with 0/0 := 0.
template <class T>
T basis_deriv(const std::vector<double>& U, int i, int k, const T& u) {
  if (k == 0) return T(0.0);
  T left(0.0), right(0.0);
  const double d1 = U[i + k] - U[i];
  const double d2 = U[i + k + 1] - U[i + 1];
  if (d1 != 0.0) left = basis(U, i, k - 1, u) * ((double)k / d1);
  if (d2 != 0.0) right = basis(U, i + 1, k - 1, u) * ((double)k / d2);
  return left - right;
}

// Knot span index i0 with u in [u_i0, u_i0+1); u = 1 goes to the last non-empty span.
int find_span(const std::vector<double>& U, int n, double u) {
  if (u >= U[n + 1]) return n;
  int i = 0;
  while (!(U[i] <= u && u < U[i + 1])) ++i;
  return i;
}

// ----------------------------------------------------------------------------
// The problem with its derived quantities.
// ----------------------------------------------------------------------------
struct Problem {
  or_problem d;
  std::vector<double> U, V;   // knot vectors in u and v
  double zmin, zmax;          // convex-hull bounds of Z (Sec. 2.1.2)
  bool two_face = false;      // freeform entry face
  std::vector<double> Uin, Vin;
  double zmin_in = 0.0, zmax_in = 0.0;
  double wx, wy;              // pixel size (Sec. 2.3)
  double Rsx, Rsy;            // effective screen radii R* with ghost pixels
  int ncol, nrow;             // extended grid: (nx+nu_x-1) columns, (ny+nu_y-1) rows
  double omega0;              // initial ray weight Phi / n_rays
  // Triangle mesh (mesh_nu > 0): the rectangles of all knot span products form
  // one uniform grid of NU x NV cells over [0,1]^2 (the knots are uniform);
  // node_z[K*(NV+1)+L] = Z(K/NU, L/NV).
  int NU = 0, NV = 0;
  std::vector<double> node_z;
};

template <class T>
void surface(const Problem& pb, const T& u, const T& v, int si, int sj, T* Z, T* Zu, T* Zv, int face = 0);

bool make_problem(const or_problem* in, Problem* pb) {
  pb->d = *in;
  const or_problem& d = pb->d;
  if (d.n1 < d.p || d.n2 < d.q || d.p < 1 || d.q < 1) return false;
  if (d.nu_x < 1 || d.nu_y < 1 || (d.nu_x % 2) == 0 || (d.nu_y % 2) == 0) return false;
  if (d.nx < 1 || d.ny < 1 || d.n_rays == 0) return false;
  pb->U = clamped_uniform_knots(d.n1, d.p);
  pb->V = clamped_uniform_knots(d.n2, d.q);
  pb->zmin = d.P[0];
  pb->zmax = d.P[0];
  for (int k = 0; k < (d.n1 + 1) * (d.n2 + 1); ++k) {
    pb->zmin = std::min(pb->zmin, d.P[k]);
    pb->zmax = std::max(pb->zmax, d.P[k]);
  }
  pb->wx = 2.0 * d.Rx / d.nx;
  pb->wy = 2.0 * d.Ry / d.ny;
  pb->Rsx = d.Rx + 0.5 * (d.nu_x - 1) * pb->wx;
  pb->Rsy = d.Ry + 0.5 * (d.nu_y - 1) * pb->wy;
  pb->ncol = d.nx + d.nu_x - 1;
  pb->nrow = d.ny + d.nu_y - 1;
  pb->omega0 = d.flux / (double)d.n_rays;
  if (d.P_in) {
    if (d.n1_in < d.p || d.n2_in < d.q || d.mesh_nu > 0) return false;
    pb->two_face = true;
    pb->Uin = clamped_uniform_knots(d.n1_in, d.p);
    pb->Vin = clamped_uniform_knots(d.n2_in, d.q);
    pb->zmin_in = pb->zmax_in = d.P_in[0];
    for (int k = 0; k < (d.n1_in + 1) * (d.n2_in + 1); ++k) {
      pb->zmin_in = std::min(pb->zmin_in, d.P_in[k]);
      pb->zmax_in = std::max(pb->zmax_in, d.P_in[k]);
    }
  }
  if (d.mesh_nu < 0 || d.mesh_nv < 0 || (d.mesh_nu > 0) != (d.mesh_nv > 0)) return false;
  if (d.mesh_nu > 0) {
    pb->NU = (d.n1 - d.p + 1) * d.mesh_nu;
    pb->NV = (d.n2 - d.q + 1) * d.mesh_nv;
    pb->node_z.assign((size_t)(pb->NU + 1) * (pb->NV + 1), 0.0);
    for (int K = 0; K <= pb->NU; ++K)
      for (int L = 0; L <= pb->NV; ++L) {
        double Z, Zu, Zv;
        surface<double>(*pb, (double)K / pb->NU, (double)L / pb->NV, -1, -1, &Z, &Zu, &Zv);
        pb->node_z[(size_t)K * (pb->NV + 1) + L] = Z;
      }
  }
  return true;
}

// Control height P^z_ij of face `face` (0 exit, 1 entry) as a T; inside the
// seeded (p+1)x(q+1) window starting at (si, sj) it carries the unit derivative
// direction (i-si)*(q+1) + (j-sj), offset by (p+1)(q+1) for the entry face.
template <class T>
T ctrl(const Problem& pb, int i, int j, int si, int sj, int face = 0) {
  const int n2 = face ? pb.d.n2_in : pb.d.n2;
  T c((face ? pb.d.P_in : pb.d.P)[i * (n2 + 1) + j]);
  const int a = i - si, b = j - sj;
  if (si >= 0 && a >= 0 && a <= pb.d.p && b >= 0 && b <= pb.d.q)
    seed_dir(c, face * (pb.d.p + 1) * (pb.d.q + 1) + a * (pb.d.q + 1) + b);
  return c;
}

// Eq. Bsplinesurfacedef for the z coordinate of face `face`, summed over every
// control point, with the first partial derivatives in u and v.
template <class T>
void surface(const Problem& pb, const T& u, const T& v, int si, int sj, T* Z, T* Zu, T* Zv, int face) {
  const int n1 = face ? pb.d.n1_in : pb.d.n1, n2 = face ? pb.d.n2_in : pb.d.n2, p = pb.d.p, q = pb.d.q;
  const std::vector<double>& U = face ? pb.Uin : pb.U;
  const std::vector<double>& V = face ? pb.Vin : pb.V;
  std::vector<T> Nu(n1 + 1), dNu(n1 + 1), Nv(n2 + 1), dNv(n2 + 1);
  for (int i = 0; i <= n1; ++i) { Nu[i] = basis(U, i, p, u); dNu[i] = basis_deriv(U, i, p, u); }
  for (int j = 0; j <= n2; ++j) { Nv[j] = basis(V, j, q, v); dNv[j] = basis_deriv(V, j, q, v); }
  T z(0.0), zu(0.0), zv(0.0);
  for (int i = 0; i <= n1; ++i) {
    for (int j = 0; j <= n2; ++j) {
      const T P = ctrl<T>(pb, i, j, si, sj, face);
      z = z + Nu[i] * Nv[j] * P;
      zu = zu + dNu[i] * Nv[j] * P;
      zv = zv + Nu[i] * dNv[j] * P;
    }
  }
  *Z = z;
  *Zu = zu;
  *Zv = zv;
}

// Z alone (used by the root scan).
double surface_z(const Problem& pb, double u, double v) {
  double Z, Zu, Zv;
  surface<double>(pb, u, v, -1, -1, &Z, &Zu, &Zv);
  return Z;
}

// X^{-1}, Y^{-1} of Sec. 2.1.1: u = (x/r_x + 1)/2, v = (y/r_y + 1)/2.
template <class T> T x_to_u(const Problem& pb, const T& x) { return (x / pb.d.rx + 1.0) * 0.5; }
template <class T> T y_to_v(const Problem& pb, const T& y) { return (y / pb.d.ry + 1.0) * 0.5; }

// ----------------------------------------------------------------------------
// Sec. 2.2: refraction and Schlick's approximation.
// ----------------------------------------------------------------------------

// Vector form of Snell's law. n_hat is the unit surface normal on the side the
// ray travels to; cos_i = d . n_hat > 0; eta = n_from / n_to. Returns false on
// total internal reflection.
template <class T>
bool refract(const T d[3], const T n[3], double eta, T t[3], T* cos_t) {
  const T ci = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
  const T k = 1.0 - eta * eta * (1.0 - ci * ci);
  if (val(k) < 0.0) return false;
  const T ct = sqrt(k);
  const T a = eta * ci - ct;
  for (int c = 0; c < 3; ++c) t[c] = eta * d[c] - a * n[c];
  *cos_t = ct;
  return true;
}

// Schlick (1994, eq. 24): R = R0 + (1-R0)(1-cos)^5 with R0 = ((n1-n2)/(n1+n2))^2,
// cos taken in the lower-index medium. Returns the transmitted fraction 1-R.
template <class T>
T schlick_transmission(double n1, double n2, const T& cos_low) {
  const double r0 = sq((n1 - n2) / (n1 + n2));
  const T c = 1.0 - cos_low;
  const T c5 = c * c * c * c * c;
  return 1.0 - (r0 + (1.0 - r0) * c5);
}

// ----------------------------------------------------------------------------
// Sec. 2.3: Gaussian reconstruction filter along one axis, over every cell of
// the extended grid: f_i = exp(-alpha ((x-c_i)/w)^2) - exp(-alpha (nu/2)^2) when
// |x-c_i| < nu w / 2, else 0, with centres c_i = (i+1/2) w - R*.
// ----------------------------------------------------------------------------
template <class T>
void filter_axis(const T& x, double Rstar, double w, int ncell, int nu, double alpha,
                 std::vector<T>& f, T* sum) {
  const double cut = std::exp(-alpha * 0.25 * nu * nu);
  T s(0.0);
  for (int i = 0; i < ncell; ++i) {
    const double c = (i + 0.5) * w - Rstar;
    const T delta = (x - c) / w;
    if (std::fabs(val(delta)) < 0.5 * nu) {
      f[i] = exp(-alpha * delta * delta) - cut;
      s = s + f[i];
    } else {
      f[i] = T(0.0);
    }
  }
  *sum = s;
}

// ----------------------------------------------------------------------------
// One ray, Secs. 2.2-2.3.
// ----------------------------------------------------------------------------
template <class T>
struct RayState {
  int status = OR_OK;
  int span_i = -1, span_j = -1;
  int span_in_i = -1, span_in_j = -1;   // freeform entry face: knot span of the entry point
  double t_in = 0.0;                     // point source, freeform entry: ray parameter of the entry point
  T u, v, x, y, z;
  T d[3];       // in-glass direction
  T tdir[3];    // direction after the freeform
  T X, Y;       // screen hit
  T w;          // final weight
  double t = 0.0;
};

// Point source: where the ray enters the glass and its direction inside.
struct GlassRay {
  int status;
  double o[3];   // entry point on z = z_in
  double d[3];   // unit direction inside the glass
  double T1;     // Schlick transmission at the entry face
};

// The ray of a point source: origin S (the source of the grid that emits it)
// and unit direction d0, uniform in the cone (Sec. 2.2.1).
void source_ray(const Problem& pb, uint64_t id, double S[3], double d0[3]);

GlassRay point_ray_in_glass(const Problem& pb, uint64_t id) {
  const or_problem& d = pb.d;
  GlassRay g{};
  double S[3], d0[3];
  source_ray(pb, id, S, d0);
  // Flat entry face z = z_in.
  const double tau = (d.z_in - S[2]) / d0[2];
  g.o[0] = S[0] + tau * d0[0];
  g.o[1] = S[1] + tau * d0[1];
  g.o[2] = d.z_in;
  if (tau <= 0.0 || std::fabs(g.o[0]) > d.rx || std::fabs(g.o[1]) > d.ry) {
    g.status = OR_APERTURE_MISS;
    return g;
  }
  const double nrm[3] = {0.0, 0.0, 1.0};
  double cos_t;
  refract<double>(d0, nrm, 1.0 / d.n_glass, g.d, &cos_t);  // never TIR into the denser medium
  g.T1 = schlick_transmission<double>(1.0, d.n_glass, d0[2]);  // cos in air = incident angle
  g.status = OR_OK;
  return g;
}

void source_ray(const Problem& pb, uint64_t id, double S[3], double d0[3]) {
  const or_problem& d = pb.d;
  double xi1, xi2;
  ray_uniforms(d.seed, id, &xi1, &xi2);
  // Which point source of the grid emits this ray (rays split evenly).
  const uint64_t n_src = (uint64_t)d.grid_nx * (uint64_t)d.grid_ny;
  const uint64_t per_src = d.n_rays / n_src;
  uint64_t s = id / per_src;
  if (s >= n_src) s = n_src - 1;
  const int sx = (int)(s % (uint64_t)d.grid_nx), sy = (int)(s / (uint64_t)d.grid_nx);
  S[0] = d.src_pos[0];
  S[1] = d.src_pos[1];
  S[2] = d.src_pos[2];
  if (d.grid_nx > 1) S[0] += -0.5 * d.grid_w + sx * d.grid_w / (d.grid_nx - 1);
  if (d.grid_ny > 1) S[1] += -0.5 * d.grid_h + sy * d.grid_h / (d.grid_ny - 1);
  // Uniform sampling of the spherical cap: theta ~ U[0,2pi), cos phi = 1-(1-cos phi_max) a.
  const double pi = 3.14159265358979323846;
  const double theta = 2.0 * pi * xi1;
  const double one_minus_cos = (1.0 - std::cos(d.half_angle)) * xi2;
  const double cos_phi = 1.0 - one_minus_cos;
  const double sin_phi = std::sqrt(one_minus_cos * (2.0 - one_minus_cos));
  d0[0] = std::cos(theta) * sin_phi;
  d0[1] = std::sin(theta) * sin_phi;
  d0[2] = cos_phi;
}

// f(t) = Z(o_uv + d_uv t) - d_z t - o_z (Eq. surfaceintersect).
double f_root(const Problem& pb, const GlassRay& g, double t) {
  double u = x_to_u<double>(pb, g.o[0] + g.d[0] * t);
  double v = y_to_v<double>(pb, g.o[1] + g.d[1] * t);
  u = std::min(1.0, std::max(0.0, u));
  v = std::min(1.0, std::max(0.0, v));
  return surface_z(pb, u, v) - g.d[2] * t - g.o[2];
}

// The smallest positive root of f on the part of the convex-hull slab
// zmin <= z <= zmax that lies over the domain [0,1]^2. A uniform scan finds the
// first sign change, then bisection narrows it to FP64 resolution.
int find_root(const Problem& pb, const GlassRay& g, double* t_root) {
  const double dz = g.d[2];
  // The slab is widened by a relative 1e-12 so that rounding in sum N_i N_j P_ij
  // cannot push Z outside it (it is degenerate for a flat freeform).
  const double pad = 1e-12 * (1.0 + std::max(std::fabs(pb.zmin), std::fabs(pb.zmax)));
  double t_lo = std::max(0.0, (pb.zmin - pad - g.o[2]) / dz);
  double t_hi = (pb.zmax + pad - g.o[2]) / dz;
  // Largest t for which the ray stays over the domain [0,1]^2.
  const double ou = x_to_u<double>(pb, g.o[0]), ov = y_to_v<double>(pb, g.o[1]);
  const double du = g.d[0] / (2.0 * pb.d.rx), dv = g.d[1] / (2.0 * pb.d.ry);
  double t_dom = INFINITY;
  if (du > 0) t_dom = std::min(t_dom, (1.0 - ou) / du);
  if (du < 0) t_dom = std::min(t_dom, (0.0 - ou) / du);
  if (dv > 0) t_dom = std::min(t_dom, (1.0 - ov) / dv);
  if (dv < 0) t_dom = std::min(t_dom, (0.0 - ov) / dv);
  if (t_dom < t_lo) return OR_OUT_OF_DOMAIN;
  const double t_end = std::min(t_hi, t_dom);
  double f_prev = f_root(pb, g, t_lo);
  if (f_prev < 0.0) return OR_INVALID;  // freeform below the entry face here
  if (f_prev == 0.0) { *t_root = t_lo; return OR_OK; }
  const int M = std::max(16, pb.d.scan_points);
  double t_prev = t_lo;
  for (int k = 1; k <= M; ++k) {
    const double t = (k == M) ? t_end : t_lo + (t_end - t_lo) * k / M;
    const double f = f_root(pb, g, t);
    if (f <= 0.0) {
      double a = t_prev, b = t;  // f(a) > 0 >= f(b)
      for (int it = 0; it < 200 && b - a > 1e-15 * std::max(1.0, b); ++it) {
        const double m = 0.5 * (a + b);
        if (f_root(pb, g, m) > 0.0) a = m; else b = m;
      }
      *t_root = 0.5 * (a + b);
      return OR_OK;
    }
    t_prev = t;
  }
  return OR_OUT_OF_DOMAIN;  // reached the side of the domain before the freeform
}

// ----------------------------------------------------------------------------
// Sec. 2.2.2: intersection with the triangle mesh of the freeform. Cell (K, L)
// is [K/NU, (K+1)/NU) x [L/NV, (L+1)/NV); with local coordinates a = NU u - K,
// b = NV v - L its lower-left triangle is {a >= 0, b >= 0, a + b < 1} and its
// upper-right triangle {a < 1, b < 1, a + b >= 1}: the paper's closed and open
// edges, which partition the cell. On each triangle the mesh is the plane
// through its three vertices on the surface (Eq. trianglefuncdetermined).
// ----------------------------------------------------------------------------
struct MeshHit {
  int status;
  int K, L, upper;
  double t;
};

// The plane of a triangle as z = c0 + ca a + cb b in the cell's local coordinates.
template <class T>
void tri_plane(const T& z00, const T& z10, const T& z01, const T& z11, int upper, T* c0, T* ca, T* cb) {
  if (!upper) {
    *c0 = z00;
    *ca = z10 - z00;
    *cb = z01 - z00;
  } else {   // z = z11 + (z11 - z01)(a - 1) + (z11 - z10)(b - 1)
    *ca = z11 - z01;
    *cb = z11 - z10;
    *c0 = z11 - *ca - *cb;
  }
}

bool in_triangle(double a, double b, int upper) {
  return upper ? (a < 1.0 && b < 1.0 && a + b >= 1.0) : (a >= 0.0 && b >= 0.0 && a + b < 1.0);
}

double node_z(const Problem& pb, int K, int L) { return pb.node_z[(size_t)K * (pb.NV + 1) + L]; }

// Mesh height at (u, v) in [0,1]^2.
double mesh_height(const Problem& pb, double u, double v) {
  const int K = std::min(pb.NU - 1, std::max(0, (int)std::floor(u * pb.NU)));
  const int L = std::min(pb.NV - 1, std::max(0, (int)std::floor(v * pb.NV)));
  const double a = u * pb.NU - K, b = v * pb.NV - L;
  double c0, ca, cb;
  tri_plane<double>(node_z(pb, K, L), node_z(pb, K + 1, L), node_z(pb, K, L + 1), node_z(pb, K + 1, L + 1),
                    a + b >= 1.0 ? 1 : 0, &c0, &ca, &cb);
  return c0 + ca * a + cb * b;
}

// Where the ray (u, v, z)(t) = (ou + du t, ov + dv t, oz + dz t) meets the plane
// of triangle (K, L, upper) with vertex heights z00, z10, z01, z11.
template <class T>
T tri_t(const Problem& pb, int K, int L, int upper, const T& z00, const T& z10, const T& z01, const T& z11,
        double ou, double ov, double oz, double du, double dv, double dz) {
  T c0, ca, cb;
  tri_plane<T>(z00, z10, z01, z11, upper, &c0, &ca, &cb);
  const double a0 = pb.NU * ou - K, b0 = pb.NV * ov - L, da = pb.NU * du, db = pb.NV * dv;
  // c0 + ca (a0 + da t) + cb (b0 + db t) = oz + dz t
  return (c0 + ca * a0 + cb * b0 - oz) / (dz - ca * da - cb * db);
}

// The first triangle the ray meets: over every triangle whose cell the ray's
// (u,v) path crosses inside the convex-hull slab, the smallest t >= 0 whose
// point lies in the triangle.
MeshHit mesh_intersect(const Problem& pb, const GlassRay& g) {
  MeshHit h{OR_OUT_OF_DOMAIN, -1, -1, 0, 0.0};
  const double dz = g.d[2];
  const double pad = 1e-12 * (1.0 + std::max(std::fabs(pb.zmin), std::fabs(pb.zmax)));
  const double t_lo = std::max(0.0, (pb.zmin - pad - g.o[2]) / dz);
  const double t_hi = (pb.zmax + pad - g.o[2]) / dz;
  const double ou = x_to_u<double>(pb, g.o[0]), ov = y_to_v<double>(pb, g.o[1]);
  const double du = g.d[0] / (2.0 * pb.d.rx), dv = g.d[1] / (2.0 * pb.d.ry);
  double t_dom = INFINITY;
  if (du > 0) t_dom = std::min(t_dom, (1.0 - ou) / du);
  if (du < 0) t_dom = std::min(t_dom, (0.0 - ou) / du);
  if (dv > 0) t_dom = std::min(t_dom, (1.0 - ov) / dv);
  if (dv < 0) t_dom = std::min(t_dom, (0.0 - ov) / dv);
  if (t_dom < t_lo) return h;
  const double t_end = std::min(t_hi, t_dom);
  auto clamp01 = [](double x) { return std::min(1.0, std::max(0.0, x)); };
  if (mesh_height(pb, clamp01(ou + du * t_lo), clamp01(ov + dv * t_lo)) - (g.o[2] + dz * t_lo) < 0.0) {
    h.status = OR_INVALID;   // freeform below the entry face here
    return h;
  }
  const double u0 = ou + du * t_lo, u1 = ou + du * t_end, v0 = ov + dv * t_lo, v1 = ov + dv * t_end;
  const int K0 = std::max(0, (int)std::floor(std::min(u0, u1) * pb.NU));
  const int K1 = std::min(pb.NU - 1, (int)std::floor(std::max(u0, u1) * pb.NU));
  const int L0 = std::max(0, (int)std::floor(std::min(v0, v1) * pb.NV));
  const int L1 = std::min(pb.NV - 1, (int)std::floor(std::max(v0, v1) * pb.NV));
  double best = INFINITY;
  for (int K = K0; K <= K1; ++K)
    for (int L = L0; L <= L1; ++L)
      for (int up = 0; up < 2; ++up) {
        const double t = tri_t<double>(pb, K, L, up, node_z(pb, K, L), node_z(pb, K + 1, L), node_z(pb, K, L + 1),
                                       node_z(pb, K + 1, L + 1), ou, ov, g.o[2], du, dv, dz);
        if (!(t >= 0.0) || !(t < best)) continue;
        if (!in_triangle(pb.NU * (ou + du * t) - K, pb.NV * (ov + dv * t) - L, up)) continue;
        best = t;
        h = MeshHit{OR_OK, K, L, up, t};
      }
  return h;
}

// A freeform entry face seen from a point source: f_in(t) = Z_in(S_uv + d0_uv t)
// - S_z - d0_z t. The entry point is its smallest positive root over the entry
// net's convex-hull slab; the ray must be over the domain [0,1]^2 at the bottom
// of the slab and stay over it until the root, else it misses the aperture (or
// meets the side of the lens first).
double f_entry(const Problem& pb, const double S[3], const double d0[3], double t) {
  double u = x_to_u<double>(pb, S[0] + d0[0] * t);
  double v = y_to_v<double>(pb, S[1] + d0[1] * t);
  u = std::min(1.0, std::max(0.0, u));
  v = std::min(1.0, std::max(0.0, v));
  double Z, Zu, Zv;
  surface<double>(pb, u, v, -1, -1, &Z, &Zu, &Zv, 1);
  return Z - d0[2] * t - S[2];
}

int find_entry_root(const Problem& pb, const double S[3], const double d0[3], double* t_root) {
  const double pad = 1e-12 * (1.0 + std::max(std::fabs(pb.zmin_in), std::fabs(pb.zmax_in)));
  const double t_lo = std::max(0.0, (pb.zmin_in - pad - S[2]) / d0[2]);
  const double t_hi = (pb.zmax_in + pad - S[2]) / d0[2];
  const double u0 = x_to_u<double>(pb, S[0] + d0[0] * t_lo), v0 = y_to_v<double>(pb, S[1] + d0[1] * t_lo);
  if (!(u0 >= 0.0 && u0 <= 1.0 && v0 >= 0.0 && v0 <= 1.0)) return OR_APERTURE_MISS;
  const double ou = x_to_u<double>(pb, S[0]), ov = y_to_v<double>(pb, S[1]);
  const double du = d0[0] / (2.0 * pb.d.rx), dv = d0[1] / (2.0 * pb.d.ry);
  double t_dom = INFINITY;
  if (du > 0) t_dom = std::min(t_dom, (1.0 - ou) / du);
  if (du < 0) t_dom = std::min(t_dom, (0.0 - ou) / du);
  if (dv > 0) t_dom = std::min(t_dom, (1.0 - ov) / dv);
  if (dv < 0) t_dom = std::min(t_dom, (0.0 - ov) / dv);
  const double t_end = std::min(t_hi, t_dom);
  double f_prev = f_entry(pb, S, d0, t_lo);
  if (f_prev < 0.0) return OR_INVALID;   // the source lies above the entry face here
  if (f_prev == 0.0) { *t_root = t_lo; return OR_OK; }
  const int M = std::max(16, pb.d.scan_points);
  double t_prev = t_lo;
  for (int k = 1; k <= M; ++k) {
    const double t = (k == M) ? t_end : t_lo + (t_end - t_lo) * k / M;
    const double f = f_entry(pb, S, d0, t);
    if (f <= 0.0) {
      double a = t_prev, b = t;
      for (int it = 0; it < 200 && b - a > 1e-15 * std::max(1.0, b); ++it) {
        const double m = 0.5 * (a + b);
        if (f_entry(pb, S, d0, m) > 0.0) a = m; else b = m;
      }
      *t_root = 0.5 * (a + b);
      return OR_OK;
    }
    t_prev = t;
  }
  return OR_APERTURE_MISS;   // left the domain through the side before entering
}

// Refraction air -> glass at a freeform entry face with slopes (Zu, Zv): the
// normal (-Z_x, -Z_y, 1)/|.| points into the glass; Schlick takes the incident
// cosine (the one in air). Never total internal reflection (into the denser medium).
template <class T>
void entry_refract(const Problem& pb, const T d0[3], const T& Zu, const T& Zv, T dg[3], T* T1) {
  const T mx = -Zu / (2.0 * pb.d.rx), my = -Zv / (2.0 * pb.d.ry);
  const T len = sqrt(mx * mx + my * my + 1.0);
  const T nrm[3] = {mx / len, my / len, 1.0 / len};
  const T ci = d0[0] * nrm[0] + d0[1] * nrm[1] + d0[2] * nrm[2];
  T cos_t;
  refract<T>(d0, nrm, 1.0 / pb.d.n_glass, dg, &cos_t);
  *T1 = schlick_transmission<T>(1.0, pb.d.n_glass, ci);
}

// Where a seeded pass starts from: the derivative windows of both faces and
// the FP64 roots of an earlier double pass of the same ray.
struct Seeds {
  int si = -1, sj = -1, si_in = -1, sj_in = -1;
  double t = 0.0, t_in = 0.0;
};

template <class T>
Seeds seeds_of(const Problem& pb, const RayState<T>& r) {
  Seeds s;
  s.si = r.span_i - pb.d.p;
  s.sj = r.span_j - pb.d.q;
  if (pb.two_face) {
    s.si_in = r.span_in_i - pb.d.p;
    s.sj_in = r.span_in_j - pb.d.q;
  }
  s.t = r.t;
  s.t_in = r.t_in;
  return s;
}

// Trace one ray. For T = double every root is found here (find_root,
// find_entry_root, mesh_intersect); for T = Dual the FP64 roots of an earlier
// double trace (in `sd`) are reused and their derivatives follow from the
// implicit function theorem applied at the root (one Newton step in dual
// arithmetic from an exact root gives dt/dP = -(df/dP)/(df/dt)).
template <class T>
void trace_ray(const Problem& pb, uint64_t id, const Seeds& sd, RayState<T>* r) {
  const or_problem& d = pb.d;
  constexpr bool is_value = std::is_same<T, double>::value;
  T T1;
  T Z, Zu, Zv;
  T o[3], dg[3];            // the ray inside the glass: origin and direction
  bool exit_root = true;    // false: a collimated ray through the flat entry face meets the exit face at (u,v)
  GlassRay g{};
  if (d.src_kind == 0) {
    // Collimated (Sec. 2.2.1): (u,v) on a square grid, direction (0,0,1).
    const uint64_t ix = id % (uint64_t)d.cols, iy = id / (uint64_t)d.cols;
    double a = 0.5, b = 0.5;
    if (d.jitter) ray_uniforms(d.seed, id, &a, &b);
    const double u = ((double)ix + a) / d.cols, v = ((double)iy + b) / d.rows;
    if (!pb.two_face) {
      // The ray starts on the freeform: its hit is (X(u), Y(v), Z(u,v)).
      r->u = T(u);
      r->v = T(v);
      r->x = (2.0 * r->u - 1.0) * d.rx;   // Eq. linearX
      r->y = (2.0 * r->v - 1.0) * d.ry;   // Eq. linearY
      r->d[0] = T(0.0); r->d[1] = T(0.0); r->d[2] = T(1.0);
      T1 = T(schlick_transmission<double>(1.0, d.n_glass, 1.0));  // normal incidence on the flat face
      surface<T>(pb, r->u, r->v, sd.si, sd.sj, &Z, &Zu, &Zv, 0);
      r->z = Z;
      exit_root = false;
    } else {
      // Freeform entry face: the ray meets it at (X(u), Y(v), Z_in(u,v)).
      T Zi, Ziu, Ziv;
      surface<T>(pb, T(u), T(v), sd.si_in, sd.sj_in, &Zi, &Ziu, &Ziv, 1);
      r->span_in_i = find_span(pb.Uin, d.n1_in, u);
      r->span_in_j = find_span(pb.Vin, d.n2_in, v);
      o[0] = T((2.0 * u - 1.0) * d.rx);
      o[1] = T((2.0 * v - 1.0) * d.ry);
      o[2] = Zi;
      const T d0[3] = {T(0.0), T(0.0), T(1.0)};
      entry_refract<T>(pb, d0, Ziu, Ziv, dg, &T1);
    }
  } else if (!pb.two_face) {
    g = point_ray_in_glass(pb, id);
    if (g.status != OR_OK) { r->status = g.status; return; }
    T1 = T(g.T1);
    for (int c = 0; c < 3; ++c) {
      o[c] = T(g.o[c]);
      dg[c] = T(g.d[c]);
    }
  } else {
    double S[3], d0[3];
    source_ray(pb, id, S, d0);
    double t_in = sd.t_in;
    if (is_value) {
      const int st = find_entry_root(pb, S, d0, &t_in);
      if (st != OR_OK) { r->status = st; return; }
    }
    r->t_in = t_in;
    T ti(t_in);
    T Zi, Ziu, Ziv;
    if (!is_value) {
      const T u0 = x_to_u<T>(pb, T(S[0] + d0[0] * t_in)), v0 = y_to_v<T>(pb, T(S[1] + d0[1] * t_in));
      surface<T>(pb, u0, v0, sd.si_in, sd.sj_in, &Zi, &Ziu, &Ziv, 1);
      const T f = Zi - d0[2] * t_in - S[2];
      const double dfdt = val(Ziu) * d0[0] / (2.0 * d.rx) + val(Ziv) * d0[1] / (2.0 * d.ry) - d0[2];
      ti = T(t_in) - f / dfdt;
    }
    for (int c = 0; c < 3; ++c) o[c] = S[c] + d0[c] * ti;
    const T ue = x_to_u<T>(pb, o[0]), ve = y_to_v<T>(pb, o[1]);
    r->span_in_i = find_span(pb.Uin, d.n1_in, std::min(1.0, std::max(0.0, val(ue))));
    r->span_in_j = find_span(pb.Vin, d.n2_in, std::min(1.0, std::max(0.0, val(ve))));
    surface<T>(pb, ue, ve, sd.si_in, sd.sj_in, &Zi, &Ziu, &Ziv, 1);
    const T d0t[3] = {T(d0[0]), T(d0[1]), T(d0[2])};
    entry_refract<T>(pb, d0t, Ziu, Ziv, dg, &T1);
  }
  if (exit_root) {
    for (int c = 0; c < 3; ++c) {
      r->d[c] = dg[c];
      g.o[c] = val(o[c]);
      g.d[c] = val(dg[c]);
    }
    double t_root = sd.t;
    MeshHit mh{};
    if (d.mesh_nu > 0) {
      // Triangle mesh (Sec. 2.2.2): the triangle is found in FP64; t is the
      // closed-form plane intersection, in T, of that triangle's vertices.
      mh = mesh_intersect(pb, g);
      if (mh.status != OR_OK) { r->status = mh.status; return; }
      t_root = mh.t;
    } else if (is_value) {
      const int st = find_root(pb, g, &t_root);
      if (st != OR_OK) { r->status = st; return; }
    }
    r->t = t_root;
    T t(t_root);
    if (d.mesh_nu > 0) {
      r->span_i = d.p + mh.K / d.mesh_nu;   // the triangle's knot span product
      r->span_j = d.q + mh.L / d.mesh_nv;
      if (!is_value) {
        T zv[4];
        for (int c = 0; c < 4; ++c) {
          T Zn, Zun, Zvn;
          surface<T>(pb, T((double)(mh.K + (c & 1)) / pb.NU), T((double)(mh.L + (c >> 1)) / pb.NV), sd.si, sd.sj,
                     &Zn, &Zun, &Zvn, 0);
          zv[c] = Zn;
        }
        const double ou = x_to_u<double>(pb, g.o[0]), ov = y_to_v<double>(pb, g.o[1]);
        t = tri_t<T>(pb, mh.K, mh.L, mh.upper, zv[0], zv[1], zv[2], zv[3], ou, ov, g.o[2],
                     g.d[0] / (2.0 * d.rx), g.d[1] / (2.0 * d.ry), g.d[2]);
      }
    } else if (!is_value) {
      const T u0 = x_to_u<T>(pb, o[0] + dg[0] * t_root);
      const T v0 = y_to_v<T>(pb, o[1] + dg[1] * t_root);
      surface<T>(pb, u0, v0, sd.si, sd.sj, &Z, &Zu, &Zv, 0);
      const T f = Z - dg[2] * t_root - o[2];
      const double dfdt = val(Zu) * g.d[0] / (2.0 * d.rx) + val(Zv) * g.d[1] / (2.0 * d.ry) - g.d[2];
      t = T(t_root) - f / dfdt;
    }
    // The hit is on the ray: o + d t.
    r->x = o[0] + dg[0] * t;
    r->y = o[1] + dg[1] * t;
    r->z = o[2] + dg[2] * t;
    r->u = x_to_u<T>(pb, r->x);
    r->v = y_to_v<T>(pb, r->y);
    surface<T>(pb, r->u, r->v, sd.si, sd.sj, &Z, &Zu, &Zv, 0);
  }
  // Knot span of the hit (for the derivative window and the records).
  if (!(d.src_kind != 0 && d.mesh_nu > 0)) {
    const double uc = std::min(1.0, std::max(0.0, val(r->u)));
    const double vc = std::min(1.0, std::max(0.0, val(r->v)));
    r->span_i = find_span(pb.U, d.n1, uc);
    r->span_j = find_span(pb.V, d.n2, vc);
  }
  // Normal of the height field z = Z(X^{-1}(x), Y^{-1}(y)) pointing into the air:
  // (-Z_x, -Z_y, 1) normalised, with Z_x = Z_u / (2 r_x), Z_y = Z_v / (2 r_y).
  const T mx = -Zu / (2.0 * d.rx), my = -Zv / (2.0 * d.ry);
  const T len = sqrt(mx * mx + my * my + 1.0);
  const T nrm[3] = {mx / len, my / len, 1.0 / len};
  T cos_t;
  if (!refract<T>(r->d, nrm, d.n_glass, r->tdir, &cos_t)) { r->status = OR_TIR; return; }
  const T T2 = schlick_transmission<T>(1.0, d.n_glass, cos_t);  // cos in air = transmitted angle
  r->w = pb.omega0 * T1 * T2;
  // Straight line to the screen z = z_screen; only rays inside the open
  // interior screen |X| < R_x, |Y| < R_y are deposited.
  if (val(r->tdir[2]) <= 0.0) { r->status = OR_OFF_SCREEN; return; }
  const T lambda = (d.z_screen - r->z) / r->tdir[2];
  r->X = r->x + lambda * r->tdir[0];
  r->Y = r->y + lambda * r->tdir[1];
  if (!(std::fabs(val(r->X)) < d.Rx && std::fabs(val(r->Y)) < d.Ry)) { r->status = OR_OFF_SCREEN; return; }
  r->status = OR_OK;
}

// The contribution w F_ij(X,Y) / (w_x w_y) of a traced ray to every pixel of
// the extended grid (Sec. 2.3), handed to `emit(col, row, value)`.
template <class T, class Emit>
void splat(const Problem& pb, const RayState<T>& r, Emit emit) {
  const or_problem& d = pb.d;
  std::vector<T> fx(pb.ncol), fy(pb.nrow);
  T sx, sy;
  filter_axis<T>(r.X, pb.Rsx, pb.wx, pb.ncol, d.nu_x, d.alpha, fx, &sx);
  filter_axis<T>(r.Y, pb.Rsy, pb.wy, pb.nrow, d.nu_y, d.alpha, fy, &sy);
  // F_ij = f_i f_j / sum_{i',j'} f_i' f_j' ; the double sum factorises. With
  // nu = 1 a ray exactly on a pixel edge has every f = 0 (the support is open):
  // the normaliser is 0/0 there and the ray deposits nothing.
  if (val(sx) == 0.0 || val(sy) == 0.0) return;
  const T scale = r.w / (sx * sy * (pb.wx * pb.wy));
  for (int j = 0; j < pb.nrow; ++j) {
    if (val(fy[j]) == 0.0) continue;
    for (int i = 0; i < pb.ncol; ++i) {
      if (val(fx[i]) == 0.0) continue;
      emit(i, j, fx[i] * fy[j] * scale);
    }
  }
}

int resolve_threads(int nthreads) {
  if (nthreads > 0) return nthreads;
  const unsigned h = std::thread::hardware_concurrency();
  return h > 0 ? (int)h : 1;
}

// Run body(thread_index, first_ray, end_ray) over `nthreads` contiguous chunks.
template <class Body>
void parallel_rays(uint64_t begin, uint64_t count, int nthreads, Body body) {
  const int nt = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)nthreads, count));
  std::vector<std::thread> pool;
  for (int k = 0; k < nt; ++k) {
    const uint64_t a = begin + count * k / nt, b = begin + count * (k + 1) / nt;
    pool.emplace_back(body, k, a, b);
  }
  for (auto& th : pool) th.join();
}

// The control heights as one parameter vector: the exit net's (n1+1)(n2+1)
// heights, then (with a freeform entry face) the entry net's.
int n_params(const Problem& pb) {
  return (pb.d.n1 + 1) * (pb.d.n2 + 1) + (pb.two_face ? (pb.d.n1_in + 1) * (pb.d.n2_in + 1) : 0);
}

// Parameter index of derivative direction c of a ray traced with seeds sd
// (directions: the exit window, then the entry window); -1 for unused ones.
int param_index(const Problem& pb, const Seeds& sd, int c) {
  const int w = (pb.d.p + 1) * (pb.d.q + 1);
  const int face = c / w, cc = c % w;
  if (face > (pb.two_face ? 1 : 0)) return -1;
  const int a2 = cc / (pb.d.q + 1), b2 = cc % (pb.d.q + 1);
  if (face == 0) return (sd.si + a2) * (pb.d.n2 + 1) + (sd.sj + b2);
  return (pb.d.n1 + 1) * (pb.d.n2 + 1) + (sd.si_in + a2) * (pb.d.n2_in + 1) + (sd.sj_in + b2);
}

// Gradient of sum_ij dLdE_ij E_ij(P) with respect to P, with NT derivative
// directions (NT >= (p+1)(q+1), twice that with a freeform entry face).
template <int NT>
void gradient_impl(const Problem& pb, uint64_t begin, uint64_t count, const double* dLdE,
                   double* dLdP, int nthreads) {
  const int nctrl = n_params(pb);
  const int nthr = resolve_threads(nthreads);
  std::vector<std::vector<double>> part(nthr, std::vector<double>(nctrl, 0.0));
  parallel_rays(begin, count, nthr, [&](int k, uint64_t a, uint64_t b) {
    std::vector<double>& g = part[k];
    for (uint64_t id = a; id < b; ++id) {
      RayState<double> r0;
      trace_ray<double>(pb, id, Seeds(), &r0);
      if (r0.status != OR_OK) continue;
      const Seeds sd = seeds_of(pb, r0);
      RayState<Dual<NT>> r;
      trace_ray<Dual<NT>>(pb, id, sd, &r);
      if (r.status != OR_OK) continue;
      double acc[NT];
      for (int c = 0; c < NT; ++c) acc[c] = 0.0;
      splat<Dual<NT>>(pb, r, [&](int i, int j, const Dual<NT>& e) {
        const double gbar = dLdE[(size_t)j * pb.ncol + i];
        if (gbar == 0.0) return;
        for (int c = 0; c < NT; ++c) acc[c] += gbar * e.d[c];
      });
      for (int c = 0; c < NT; ++c) {
        const int pi = param_index(pb, sd, c);
        if (pi >= 0) g[pi] += acc[c];
      }
    }
  });
  for (int c = 0; c < nctrl; ++c) dLdP[c] = 0.0;
  for (int k = 0; k < nthr; ++k)
    for (int c = 0; c < nctrl; ++c) dLdP[c] += part[k][c];
}

// Directional derivatives dE = (dE/dP^z) dP_k of the irradiance for n_dirs
// directions dP_k (forward mode: the same per-ray dual numbers as the gradient,
// contracted with each direction instead of with dL/dE).
template <int NT>
void tangent_impl(const Problem& pb, uint64_t begin, uint64_t count, const double* dP, int n_dirs, double* dE,
                  int nthreads) {
  const int nctrl = n_params(pb);
  const size_t ncell = (size_t)pb.ncol * pb.nrow;
  const int nthr = resolve_threads(nthreads);
  std::vector<std::vector<double>> part(nthr, std::vector<double>(ncell * n_dirs, 0.0));
  parallel_rays(begin, count, nthr, [&](int k, uint64_t a, uint64_t b) {
    std::vector<double>& e = part[k];
    std::vector<double> local((size_t)n_dirs * NT);
    for (uint64_t id = a; id < b; ++id) {
      RayState<double> r0;
      trace_ray<double>(pb, id, Seeds(), &r0);
      if (r0.status != OR_OK) continue;
      const Seeds sd = seeds_of(pb, r0);
      bool any = false;
      for (int q = 0; q < n_dirs; ++q)
        for (int c = 0; c < NT; ++c) {
          const int pi = param_index(pb, sd, c);
          const double v = pi >= 0 ? dP[(size_t)q * nctrl + pi] : 0.0;
          local[(size_t)q * NT + c] = v;
          any = any || v != 0.0;
        }
      if (!any) continue;
      RayState<Dual<NT>> r;
      trace_ray<Dual<NT>>(pb, id, sd, &r);
      if (r.status != OR_OK) continue;
      splat<Dual<NT>>(pb, r, [&](int i, int j, const Dual<NT>& ed) {
        for (int q = 0; q < n_dirs; ++q) {
          double v = 0.0;
          for (int c = 0; c < NT; ++c) v += ed.d[c] * local[(size_t)q * NT + c];
          e[(size_t)q * ncell + (size_t)j * pb.ncol + i] += v;
        }
      });
    }
  });
  for (size_t c = 0; c < ncell * n_dirs; ++c) dE[c] = 0.0;
  for (int k = 0; k < nthr; ++k)
    for (size_t c = 0; c < ncell * n_dirs; ++c) dE[c] += part[k][c];
}

}  // namespace

// ----------------------------------------------------------------------------
// C entry points (loaded by oracle/oracle.py through ctypes).
// Return 0 on success, -1 on an invalid problem.
// ----------------------------------------------------------------------------
extern "C" {

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  philox4x32_10(ctr, key, out);
}

void or_ray_uniforms(uint64_t seed, uint64_t id, double* xi1, double* xi2) {
  ray_uniforms(seed, id, xi1, xi2);
}

// Knot vector (n+p+2 entries) of the clamped uniform B-spline.
void or_knots(int32_t n, int32_t p, double* out) {
  const std::vector<double> U = clamped_uniform_knots(n, p);
  for (size_t k = 0; k < U.size(); ++k) out[k] = U[k];
}

// All n+1 basis values N_{i,p}(u) and first derivatives at u.
void or_basis(int32_t n, int32_t p, double u, double* N, double* dN) {
  const std::vector<double> U = clamped_uniform_knots(n, p);
  for (int i = 0; i <= n; ++i) {
    N[i] = basis<double>(U, i, p, u);
    dN[i] = basis_deriv<double>(U, i, p, u);
  }
}

// Z, Z_u, Z_v at (u,v) and the second derivatives by the same code in dual
// arithmetic (direction 0 = u, 1 = v): out = {Z, Zu, Zv, Zuu, Zuv, Zvv}.
int32_t or_surface(const or_problem* prob, double u, double v, double* out) {
  Problem pb;
  if (!make_problem(prob, &pb)) return -1;
  Dual<2> ud(u), vd(v);
  ud.d[0] = 1.0;
  vd.d[1] = 1.0;
  Dual<2> Z, Zu, Zv;
  surface<Dual<2>>(pb, ud, vd, -1, -1, &Z, &Zu, &Zv);
  out[0] = Z.v; out[1] = Zu.v; out[2] = Zv.v;
  out[3] = Zu.d[0]; out[4] = Zu.d[1]; out[5] = Zv.d[1];
  return 0;
}

// Vector Snell law; returns 1 on total internal reflection.
int32_t or_refract(const double d[3], const double n[3], double eta, double t[3], double* cos_t) {
  return refract<double>(d, n, eta, t, cos_t) ? 0 : 1;
}

double or_schlick_transmission(double n1, double n2, double cos_low) {
  return schlick_transmission<double>(n1, n2, cos_low);
}

// Filter values f_i along one axis over every cell, and their sum.
void or_filter_axis(double x, double Rstar, double w, int32_t ncell, int32_t nu, double alpha,
                    double* f, double* sum) {
  std::vector<double> fv(ncell);
  filter_axis<double>(x, Rstar, w, ncell, nu, alpha, fv, sum);
  for (int i = 0; i < ncell; ++i) f[i] = fv[i];
}

// Direction of a point-source ray and where it enters the glass.
int32_t or_point_ray(const or_problem* prob, uint64_t id, double o[3], double d[3], double* T1) {
  Problem pb;
  if (!make_problem(prob, &pb)) return -1;
  const GlassRay g = point_ray_in_glass(pb, id);
  for (int c = 0; c < 3; ++c) { o[c] = g.o[c]; d[c] = g.d[c]; }
  *T1 = g.T1;
  return g.status;
}

// Per-ray records of rays [begin, begin+count).
int32_t or_trace_records(const or_problem* prob, uint64_t begin, uint64_t count, or_record* out,
                         int32_t nthreads) {
  Problem pb;
  if (!make_problem(prob, &pb)) return -1;
  parallel_rays(begin, count, resolve_threads(nthreads), [&](int, uint64_t a, uint64_t b) {
    for (uint64_t id = a; id < b; ++id) {
      RayState<double> r;
      trace_ray<double>(pb, id, Seeds(), &r);
      or_record& o = out[id - begin];
      std::memset(&o, 0, sizeof o);
      o.status = r.status;
      o.span_i = r.span_i;
      o.span_j = r.span_j;
      if (r.status == OR_APERTURE_MISS) continue;
      o.dx = r.d[0]; o.dy = r.d[1]; o.dz = r.d[2];
      o.t = r.t;
      if (r.status == OR_OUT_OF_DOMAIN || r.status == OR_INVALID) continue;
      o.u = r.u; o.v = r.v; o.x = r.x; o.y = r.y; o.z = r.z;
      if (r.status == OR_TIR) continue;
      o.tx = r.tdir[0]; o.ty = r.tdir[1]; o.tz = r.tdir[2];
      o.w = r.w;
      if (r.status == OR_OFF_SCREEN) continue;
      o.X = r.X; o.Y = r.Y;
    }
  });
  return 0;
}

// Irradiance of rays [begin, begin+count) on the extended grid
// ((ny+nu_y-1) rows x (nx+nu_x-1) columns, row-major), and counts per status.
int32_t or_trace_forward(const or_problem* prob, uint64_t begin, uint64_t count, double* E,
                         or_stats* stats, int32_t nthreads) {
  Problem pb;
  if (!make_problem(prob, &pb)) return -1;
  const size_t ncell = (size_t)pb.ncol * pb.nrow;
  const int nthr = resolve_threads(nthreads);
  std::vector<std::vector<double>> part(nthr, std::vector<double>(ncell, 0.0));
  std::vector<or_stats> st(nthr);
  for (auto& s : st) std::memset(&s, 0, sizeof s);
  parallel_rays(begin, count, nthr, [&](int k, uint64_t a, uint64_t b) {
    std::vector<double>& e = part[k];
    for (uint64_t id = a; id < b; ++id) {
      RayState<double> r;
      trace_ray<double>(pb, id, Seeds(), &r);
      st[k].counts[r.status] += 1;
      if (r.status != OR_OK) continue;
      splat<double>(pb, r, [&](int i, int j, double c) { e[(size_t)j * pb.ncol + i] += c; });
    }
  });
  for (size_t c = 0; c < ncell; ++c) E[c] = 0.0;
  for (int k = 0; k < nthr; ++k)
    for (size_t c = 0; c < ncell; ++c) E[c] += part[k][c];
  if (stats) {
    std::memset(stats, 0, sizeof *stats);
    for (int k = 0; k < nthr; ++k)
      for (int c = 0; c < 8; ++c) stats->counts[c] += st[k].counts[c];
  }
  return 0;
}

// dL/dP^z = sum over rays [begin, begin+count) and pixels of dL/dE_ij dE_ij/dP^z,
// with dLdE on the extended grid.
int32_t or_trace_gradient(const or_problem* prob, uint64_t begin, uint64_t count, const double* dLdE,
                          double* dLdP, int32_t nthreads) {
  Problem pb;
  if (!make_problem(prob, &pb)) return -1;
  const int ndir = (pb.d.p + 1) * (pb.d.q + 1) * (pb.two_face ? 2 : 1);
  if (ndir <= 16) gradient_impl<16>(pb, begin, count, dLdE, dLdP, nthreads);
  else if (ndir <= 36) gradient_impl<36>(pb, begin, count, dLdE, dLdP, nthreads);
  else return -1;
  return 0;
}

// dE_k = (dE/dP^z) dP_k over rays [begin, begin+count) for n_dirs directions
// (dP: n_dirs x (n1+1)(n2+1); dE: n_dirs extended grids).
int32_t or_trace_tangent(const or_problem* prob, uint64_t begin, uint64_t count, const double* dP, int32_t n_dirs,
                         double* dE, int32_t nthreads) {
  Problem pb;
  if (!make_problem(prob, &pb) || n_dirs < 1) return -1;
  const int ndir = (pb.d.p + 1) * (pb.d.q + 1) * (pb.two_face ? 2 : 1);
  if (ndir <= 16) tangent_impl<16>(pb, begin, count, dP, n_dirs, dE, nthreads);
  else if (ndir <= 36) tangent_impl<36>(pb, begin, count, dP, n_dirs, dE, nthreads);
  else return -1;
  return 0;
}

// Squared L2 loss over the interior pixels, L = sum (E - E_ref)^2, and
// dL/dE = 2 (E - E_ref) on the interior (0 on ghost pixels). E and dLdE are on
// the extended grid, E_ref on the interior ny x nx grid.
double or_loss_l2(const double* E, const double* E_ref, int32_t nx, int32_t ny, int32_t nu_x, int32_t nu_y,
                  double* dLdE) {
  const int hx = (nu_x - 1) / 2, hy = (nu_y - 1) / 2;
  const int ncol = nx + nu_x - 1, nrow = ny + nu_y - 1;
  for (int c = 0; c < ncol * nrow; ++c) dLdE[c] = 0.0;
  double L = 0.0;
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i < nx; ++i) {
      const double diff = E[(size_t)(j + hy) * ncol + (i + hx)] - E_ref[(size_t)j * nx + i];
      L += diff * diff;
      dLdE[(size_t)(j + hy) * ncol + (i + hx)] = 2.0 * diff;
    }
  }
  return L;
}

// The paper's loss (Sec. 2.5): with I^ = I / sum(I) and I^_ref = I_ref / sum(I_ref)
// over the nx x ny interior, L = ||I^ - I^_ref||_F / sqrt(nx ny). dLdE (extended
// grid) gets dL/dI on the interior and 0 on ghost pixels. By the chain rule through
// I^_kl = I_kl / S (S = sum I): dL/dI_ij = (g_ij - sum_kl g_kl I^_kl) / S, where
// g = dL/dI^ = (I^ - I^_ref) / (sqrt(nx ny) ||I^ - I^_ref||_F).
// Where the norm is 0 (images equal up to scale) the gradient is taken as 0.
// Where S or sum(I_ref) is not positive the normalisation is undefined: the loss
// is NaN and the gradient 0.
double or_loss_frobenius(const double* E, const double* E_ref, int32_t nx, int32_t ny, int32_t nu_x, int32_t nu_y,
                         double* dLdE) {
  const int hx = (nu_x - 1) / 2, hy = (nu_y - 1) / 2;
  const int ncol = nx + nu_x - 1, nrow = ny + nu_y - 1;
  for (int c = 0; c < ncol * nrow; ++c) dLdE[c] = 0.0;
  auto I = [&](int i, int j) { return E[(size_t)(j + hy) * ncol + (i + hx)]; };
  double S = 0.0, Sref = 0.0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      S += I(i, j);
      Sref += E_ref[(size_t)j * nx + i];
    }
  if (!(S > 0.0) || !(Sref > 0.0)) return std::nan("");
  std::vector<double> D((size_t)nx * ny);
  double norm2 = 0.0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const double d = I(i, j) / S - E_ref[(size_t)j * nx + i] / Sref;
      D[(size_t)j * nx + i] = d;
      norm2 += d * d;
    }
  const double root_n = std::sqrt((double)nx * (double)ny);
  const double norm = std::sqrt(norm2);
  const double L = norm / root_n;
  if (norm == 0.0) return L;
  double gdot = 0.0;                        // sum_kl g_kl I^_kl
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) gdot += D[(size_t)j * nx + i] / (root_n * norm) * (I(i, j) / S);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const double g = D[(size_t)j * nx + i] / (root_n * norm);
      dLdE[(size_t)(j + hy) * ncol + (i + hx)] = (g - gdot) / S;
    }
  return L;
}

// Greville abscissae u*_i = (u_{i+1} + ... + u_{i+p}) / p, i = 0..n, of the clamped
// uniform knot vector (Sec. 2.1, Farin sec. 8.6).
void or_greville(int32_t n, int32_t p, double* out) {
  const std::vector<double> U = clamped_uniform_knots(n, p);
  for (int i = 0; i <= n; ++i) {
    double s = 0.0;
    for (int k = i + 1; k <= i + p; ++k) s += U[k];
    out[i] = s / p;
  }
}

// Offset f(P^x_ij, P^y_ij) at the control points, P^x_ij = (2u*_i - 1) r_x and
// P^y_ij = (2v*_j - 1) r_y (Greville construction, Sec. 2.1). f is the spherical
// cap of Table magndata: f = c + R - sign(R) sqrt(R^2 - x^2 - y^2), a sphere of
// radius |R| through (0, 0, c); R = 0 gives the constant c. Returns -1 if a
// control point lies outside the sphere's footprint (x^2 + y^2 > R^2).
int32_t or_offset_spherical(int32_t n1, int32_t n2, int32_t p, int32_t q, double rx, double ry, double c, double R,
                            double* out) {
  std::vector<double> gu(n1 + 1), gv(n2 + 1);
  or_greville(n1, p, gu.data());
  or_greville(n2, q, gv.data());
  for (int i = 0; i <= n1; ++i)
    for (int j = 0; j <= n2; ++j) {
      const double x = (2.0 * gu[i] - 1.0) * rx, y = (2.0 * gv[j] - 1.0) * ry;
      double f = c;
      if (R != 0.0) {
        const double r2 = R * R - x * x - y * y;
        if (r2 < 0.0) return -1;
        f = c + R - (R > 0.0 ? 1.0 : -1.0) * std::sqrt(r2);
      }
      out[(size_t)i * (n2 + 1) + j] = f;
    }
  return 0;
}

// Control heights from unconstrained variables (Sec. 2.4.2): P_k = offset_k +
// z_min + (tanh(theta_k) + 1)(z_max - z_min)/2; offset may be NULL (= 0).
void or_reparam_tanh(const double* theta, const double* offset, int32_t n, double z_min, double z_max, double* P) {
  for (int k = 0; k < n; ++k)
    P[k] = (offset ? offset[k] : 0.0) + z_min + 0.5 * (std::tanh(theta[k]) + 1.0) * (z_max - z_min);
}

// Its adjoint: dL/dtheta_k = dL/dP_k (z_max - z_min)/2 (1 - tanh^2(theta_k)).
void or_reparam_tanh_adjoint(const double* theta, const double* dLdP, int32_t n, double z_min, double z_max,
                             double* dLdtheta) {
  for (int k = 0; k < n; ++k) {
    const double t = std::tanh(theta[k]);
    dLdtheta[k] = dLdP[k] * 0.5 * (z_max - z_min) * (1.0 - t * t);
  }
}

// Adam (Kingma & Ba, Algorithm 1), step number `step` counted from 1.
void or_adam_step(double* theta, double* m, double* v, const double* g, int32_t n, double lr, double beta1,
                  double beta2, double eps, int32_t step) {
  for (int k = 0; k < n; ++k) {
    m[k] = beta1 * m[k] + (1.0 - beta1) * g[k];
    v[k] = beta2 * v[k] + (1.0 - beta2) * g[k] * g[k];
    const double mhat = m[k] / (1.0 - std::pow(beta1, step));
    const double vhat = v[k] / (1.0 - std::pow(beta2, step));
    theta[k] -= lr * mhat / (std::sqrt(vhat) + eps);
  }
}

}  // extern "C"
