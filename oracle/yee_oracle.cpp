// FP64 CPU oracle for the time-reversible Yee FDTD hot path.
//
// TEST INFRASTRUCTURE ONLY. This file is the plain, slow reference that the CUDA path is checked
// against. Nothing in the product path links, loads or calls it; only tests/, the smoke check and
// the bench's CPU-baseline leg do. It shares no code with the CUDA library.
//
// What it computes (arXiv 2412.12360, "FDTDX"):
//   * Sec. 2.1, Eqs. (1)-(2): Faraday and Ampere curl updates on the Yee grid, repeated per time step,
//     with a convolutional PML (CPML, the Roden-Gedney form cited in Sec. 2.1) on the outer faces,
//     soft sources, and detectors that record fields at intermediate steps (interpolation off).
//   * Sec. 2.2: the reverse-mode derivative of the discrete forward map, obtained three ways:
//       - store every intermediate state (the plain automatic-differentiation baseline of Sec. 2.2),
//       - fixed-interval checkpointing with recomputation (a simple member of the checkpointing family
//         of Sec. 2.2),
//       - time reversal: the inverse update step t+1 -> t of Sec. 2.2, with the fields on the boundary
//         between the PML and the inner volume recorded every step and replayed ("six two-dimensional
//         slices").
//   * a complex-step derivative through a templated scalar, as an independent check of the adjoint.
//
// Readings where the paper gives no formula (it prints only Eqs. 1-2):
//   normalised units c = 1, dx = 1, H~ = eta0 H, mu = 1; S = c dt / dx is the Courant number; one
//   inverse permittivity a = 1/eps per cell, shared by that cell's Ex, Ey, Ez; PEC at integer planes
//   0 and N on every axis; CPML with polynomial grading sigma = sigma_max (d/p)^m, kappa = 1 +
//   (kappa_max - 1)(d/p)^m, alpha = alpha_max (1 - d/p), b = exp(-(sigma/kappa + alpha)),
//   c = sigma/(sigma kappa + kappa^2 alpha) (b - 1), d the depth of the component's own position
//   into the layer; source waveform g(s) = sin(2 pi (s - t0)/P) exp(-((s - t0)/tau)^2), P = lambda/S
//   steps, sampled at s = n + 1/2 and added to E after the E update; detectors sample E^{n+1} and
//   H^{n+1/2} after every step.
//
// Build: g++ -O2 -std=c++17 -fopenmp -ffp-contract=off -shared -fPIC (no FMA contraction).

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

extern "C" {

// A source on an E component over a box of cells [lo, hi): a soft source (tfsf = 0), or the plane of
// a one-sided total-field / scattered-field source (tfsf = +-(axis + 1), the sign giving the direction
// of travel; the box is one cell thick along the axis).
typedef struct {
  int32_t component;      // 0, 1, 2 = Ex, Ey, Ez
  int32_t lo[3], hi[3];   // cell box, x fastest
  const double* profile;  // box-shaped weights (x fastest), or NULL for 1 everywhere
  double amplitude;
  double wavelength_cells;
  double tau_steps;       // width of the Gaussian envelope, in steps
  double t0_steps;        // centre of the envelope, in steps
  int32_t tfsf;
  double eps_background;  // TFSF: permittivity of the one-dimensional incident-field line
} orc_source;

// Detector kinds. Outputs are concatenated in detector order.
//   0 point series : value of field `component` (0..5 = Ex..Hz) at cell lo, one value per step.
//   1 |E|^2 sum    : per cell of the box, sum over steps of Ex^2 + Ey^2 + Ez^2 (same-index samples).
//   2 flux series  : per step, sum over the box of (E x H)[axis] (same-index samples).
// With interpolation (Sec. 2.1: composite metrics need the staggered components brought to one point
// in space and time; the paper's evaluation mode), every component is taken at the cell centre
// (i+1/2, j+1/2, k+1/2): E_c as the mean of its 4 values around the centre (offsets 0/1 along the two
// axes other than c), H_c as the mean of its 2 values (offsets 0/1 along c); values beyond the grid
// are 0 (the box plus one cell must lie in the grid).
//   3 |E|^2 sum, interpolated : per cell, sum over steps of |E^{n+1}(centre)|^2;
//   4 flux series, interpolated: per step, sum over the box of (E^{n+1/2} x H^{n+1/2})[axis] at the
//     centres, E^{n+1/2} = (E^n + E^{n+1}) / 2.
typedef struct {
  int32_t kind;
  int32_t component;
  int32_t axis;
  int32_t lo[3], hi[3];
} orc_detector;

typedef struct {
  int32_t n[3];           // cells along x, y, z
  double courant;         // S = c dt / dx
  int32_t pml[6];         // layer thickness in cells: x-lo, x-hi, y-lo, y-hi, z-lo, z-hi (0 = PEC wall)
  double sigma_max, kappa_max, alpha_max;
  int32_t grading_m;
  const double* eps_inv;  // n[2]*n[1]*n[0], x fastest
  int32_t nsrc;
  const orc_source* src;
  int32_t ndet;
  const orc_detector* det;
  int32_t design_lo[3], design_hi[3];
} orc_scene;

}  // extern "C"

namespace {

typedef std::complex<double> cplx;

inline int m3(int c) { return c % 3; }

struct Geometry {
  int n[3];
  size_t N;
  explicit Geometry(const orc_scene& s) {
    for (int d = 0; d < 3; ++d) n[d] = s.n[d];
    N = size_t(n[0]) * n[1] * n[2];
  }
  size_t at(int i, int j, int k) const { return (size_t(k) * n[1] + j) * n[0] + i; }
  size_t at(const int* p) const { return at(p[0], p[1], p[2]); }
};

// CPML coefficients for one axis, at integer positions (index i) and half positions (index i + 1/2).
struct AxisCoef {
  std::vector<double> b_int, c_int, kappa_int, b_half, c_half, kappa_half;
};

void grade(const orc_scene& s, int axis, double x, double& b, double& c, double& kappa) {
  const int N = s.n[axis], p0 = s.pml[2 * axis], p1 = s.pml[2 * axis + 1];
  double d = 0.0;
  if (p0 > 0 && x < p0) d = (p0 - x) / p0;
  else if (p1 > 0 && x > N - p1) d = (x - (N - p1)) / p1;
  if (d <= 0.0) { b = 1.0; c = 0.0; kappa = 1.0; return; }
  const double dm = std::pow(d, s.grading_m);
  const double sigma = s.sigma_max * dm;
  kappa = 1.0 + (s.kappa_max - 1.0) * dm;
  const double alpha = s.alpha_max * (1.0 - d);
  b = std::exp(-(sigma / kappa + alpha));
  c = (sigma == 0.0) ? 0.0 : sigma / (sigma * kappa + kappa * kappa * alpha) * (b - 1.0);
}

std::vector<AxisCoef> make_coefs(const orc_scene& s) {
  std::vector<AxisCoef> ax(3);
  for (int d = 0; d < 3; ++d) {
    const int N = s.n[d];
    AxisCoef& a = ax[d];
    a.b_int.resize(N); a.c_int.resize(N); a.kappa_int.resize(N);
    a.b_half.resize(N); a.c_half.resize(N); a.kappa_half.resize(N);
    for (int i = 0; i < N; ++i) {
      grade(s, d, double(i), a.b_int[i], a.c_int[i], a.kappa_int[i]);
      grade(s, d, i + 0.5, a.b_half[i], a.c_half[i], a.kappa_half[i]);
    }
  }
  return ax;
}

double waveform(const orc_source& src, double S, double s) {
  const double P = src.wavelength_cells / S;
  const double u = s - src.t0_steps;
  return std::sin(2.0 * M_PI * u / P) * std::exp(-(u / src.tau_steps) * (u / src.tau_steps));
}

// Total-field / scattered-field plane source (Sec. 2.1: the incident field enters on one side only).
// The incident plane wave (E component c, H component h, travelling along `axis` in direction dir)
// comes from a one-dimensional Yee line along the axis with the same S and a = 1/eps_background,
// driven by a soft source amplitude * g(n + 1/2) on its E a few cells upstream of the plane. Its
// equations are the 3-D ones restricted to the axis: (curl H)_c holds sE dH_h/d(axis) and
// (curl E)_h holds sH dE_c/d(axis), with sE, sH = +-1 from the cyclic order of the components.
// The plane's E_c (index k) is total field, the adjacent H_h (index k-1 when dir > 0, k when dir < 0)
// scattered field; each side's update reads one value of the other side, so it gets the incident
// value as a correction:
//   H_h += dir S sH Einc^n(k)                 after the H update of step n,
//   E_c += -dir S a sE Hinc^{n+1/2}(k -+ 1/2)  after the E update of step n.
struct Tfsf {
  int axis = 0, dir = 0, c = 0, h = 0, hidx = 0;
  double sE = 0, sH = 0;
  std::vector<double> einc, hinc;  // Einc^n at the plane, Hinc^{n+1/2} at the adjacent H plane
};

Tfsf make_tfsf(const orc_source& s, double S, int nsteps) {
  Tfsf t;
  t.axis = std::abs(s.tfsf) - 1;
  t.dir = s.tfsf > 0 ? 1 : -1;
  t.c = s.component;
  t.h = 3 - t.axis - t.c;
  t.sE = (t.axis == m3(t.c + 1)) ? 1.0 : -1.0;  // (curl H)_c = dH_{c+2}/dx_{c+1} - dH_{c+1}/dx_{c+2}
  t.sH = (t.axis == m3(t.h + 1)) ? 1.0 : -1.0;  // (curl E)_h = dE_{h+2}/dx_{h+1} - dE_{h+1}/dx_{h+2}
  t.hidx = s.lo[t.axis] - (t.dir > 0 ? 1 : 0);
  const int L = 2 * nsteps + 16, K = nsteps + 8, ksrc = K - 4 * t.dir;
  const double ab = 1.0 / s.eps_background;
  std::vector<double> E(L, 0.0), H(L, 0.0);  // H[k] sits at k + 1/2; E[0] is a PEC end
  t.einc.resize(nsteps);
  t.hinc.resize(nsteps);
  for (int n = 0; n < nsteps; ++n) {
    t.einc[n] = E[K];
    for (int k = 0; k + 1 < L; ++k) H[k] -= S * t.sH * (E[k + 1] - E[k]);
    t.hinc[n] = t.dir > 0 ? H[K - 1] : H[K];
    for (int k = 1; k < L; ++k) E[k] += S * ab * t.sE * (H[k] - H[k - 1]);
    E[ksrc] += s.amplitude * waveform(s, S, n + 0.5);
  }
  return t;
}

template <class T>
struct State {
  std::vector<T> F[6];           // Ex, Ey, Ez, Hx, Hy, Hz
  std::vector<T> psiE[3][3];     // psiE[c][d]: CPML memory of E_c for the derivative along d != c
  std::vector<T> psiH[3][3];
  explicit State(size_t N = 0) { resize(N); }
  void resize(size_t N) {
    for (int f = 0; f < 6; ++f) F[f].assign(N, T(0));
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) {
        psiE[c][d].assign(c == d ? 0 : N, T(0));
        psiH[c][d].assign(c == d ? 0 : N, T(0));
      }
  }
};

// Everything the time loop needs, built once per call.
template <class T>
struct Sim {
  const orc_scene& sc;
  Geometry g;
  double S;
  std::vector<AxisCoef> cf;
  std::vector<T> a;                 // inverse permittivity per cell (T so a complex step can perturb it)
  std::vector<size_t> det_offset;   // start of each detector's output in the concatenated vector
  size_t det_total = 0;
  int nsteps;
  std::vector<Tfsf> tfsf;           // per source (used where the source has tfsf != 0)
  bool time_interp = false;         // some detector needs E^n beside E^{n+1} (kind 4)
  mutable std::vector<T> prevE[3];  // E^n of the step being sampled (kind 4 only)

  Sim(const orc_scene& s, int nsteps_) : sc(s), g(s), S(s.courant), cf(make_coefs(s)), nsteps(nsteps_) {
    a.resize(g.N);
    for (size_t p = 0; p < g.N; ++p) a[p] = T(s.eps_inv[p]);
    tfsf.resize(s.nsrc);
    for (int q = 0; q < s.nsrc; ++q)
      if (s.src[q].tfsf != 0) tfsf[q] = make_tfsf(s.src[q], S, nsteps);
    for (int q = 0; q < s.ndet; ++q) time_interp = time_interp || s.det[q].kind == 4;
    for (int q = 0; q < s.ndet; ++q) {
      det_offset.push_back(det_total);
      det_total += det_size(s.det[q]);
    }
  }
  size_t det_size(const orc_detector& d) const {
    if (d.kind == 1 || d.kind == 3)
      return size_t(d.hi[0] - d.lo[0]) * (d.hi[1] - d.lo[1]) * (d.hi[2] - d.lo[2]);
    return size_t(nsteps);
  }

  // E is updated unless it is tangential to a PEC wall at index 0 of one of its two transverse axes.
  bool e_updated(int c, const int* p) const { return p[m3(c + 1)] != 0 && p[m3(c + 2)] != 0; }

  // ---- Sec. 2.1, Eq. (1): H^{n+1/2} = H^{n-1/2} - S curl E^n, with CPML -------------------------
  void update_H(State<T>& st) const {
    for (int c = 0; c < 3; ++c) {
      const int c1 = m3(c + 1), c2 = m3(c + 2);
      std::vector<T>& H = st.F[3 + c];
      const std::vector<T>& Ea = st.F[c2];  // differenced along c1
      const std::vector<T>& Eb = st.F[c1];  // differenced along c2
#pragma omp parallel for
      for (int k = 0; k < g.n[2]; ++k)
        for (int j = 0; j < g.n[1]; ++j)
          for (int i = 0; i < g.n[0]; ++i) {
            int p[3] = {i, j, k};
            const size_t q = g.at(p);
            int p1[3] = {i, j, k}; p1[c1] += 1;
            int p2[3] = {i, j, k}; p2[c2] += 1;
            const T ea1 = (p1[c1] < g.n[c1]) ? Ea[g.at(p1)] : T(0);  // index N lies on the PEC wall
            const T eb2 = (p2[c2] < g.n[c2]) ? Eb[g.at(p2)] : T(0);
            const T d1 = ea1 - Ea[q];
            const T d2 = eb2 - Eb[q];
            const AxisCoef& A1 = cf[c1];
            const AxisCoef& A2 = cf[c2];
            T& s1 = st.psiH[c][c1][q];
            T& s2 = st.psiH[c][c2][q];
            s1 = A1.b_half[p[c1]] * s1 + A1.c_half[p[c1]] * d1;
            s2 = A2.b_half[p[c2]] * s2 + A2.c_half[p[c2]] * d2;
            H[q] -= S * (d1 / A1.kappa_half[p[c1]] + s1 - d2 / A2.kappa_half[p[c2]] - s2);
          }
    }
  }

  // ---- Sec. 2.1, Eq. (2): E^{n+1} = E^n + S a curl H^{n+1/2}, with CPML ------------------------
  void update_E(State<T>& st) const {
    for (int c = 0; c < 3; ++c) {
      const int c1 = m3(c + 1), c2 = m3(c + 2);
      std::vector<T>& E = st.F[c];
      const std::vector<T>& Ha = st.F[3 + c2];  // differenced along c1
      const std::vector<T>& Hb = st.F[3 + c1];  // differenced along c2
#pragma omp parallel for
      for (int k = 0; k < g.n[2]; ++k)
        for (int j = 0; j < g.n[1]; ++j)
          for (int i = 0; i < g.n[0]; ++i) {
            int p[3] = {i, j, k};
            if (!e_updated(c, p)) continue;
            const size_t q = g.at(p);
            int p1[3] = {i, j, k}; p1[c1] -= 1;
            int p2[3] = {i, j, k}; p2[c2] -= 1;
            const T d1 = Ha[q] - Ha[g.at(p1)];
            const T d2 = Hb[q] - Hb[g.at(p2)];
            const AxisCoef& A1 = cf[c1];
            const AxisCoef& A2 = cf[c2];
            T& s1 = st.psiE[c][c1][q];
            T& s2 = st.psiE[c][c2][q];
            s1 = A1.b_int[p[c1]] * s1 + A1.c_int[p[c1]] * d1;
            s2 = A2.b_int[p[c2]] * s2 + A2.c_int[p[c2]] * d2;
            E[q] += S * a[q] * (d1 / A1.kappa_int[p[c1]] + s1 - d2 / A2.kappa_int[p[c2]] - s2);
          }
    }
  }

  // E sources after the E update of step n: soft sources E_c += amplitude * profile * g(n + 1/2);
  // the E correction of a TFSF plane, -dir S a sE profile Hinc^{n+1/2} (a of the cell, held constant:
  // the plane lies outside the design box). With only_R, cells outside R are skipped.
  void add_sources(State<T>& st, int n, double sign, bool only_R = false) const {
    for (int q = 0; q < sc.nsrc; ++q) {
      const orc_source& s = sc.src[q];
      const Tfsf& t = tfsf[q];
      const double gn = s.tfsf ? -t.dir * S * t.sE * t.hinc[n] : s.amplitude * waveform(s, S, n + 0.5);
      const int bx = s.hi[0] - s.lo[0], by = s.hi[1] - s.lo[1];
      for (int k = s.lo[2]; k < s.hi[2]; ++k)
        for (int j = s.lo[1]; j < s.hi[1]; ++j)
          for (int i = s.lo[0]; i < s.hi[0]; ++i) {
            int p[3] = {i, j, k};
            if (!e_updated(s.component, p)) continue;
            if (only_R && !e_in_R(s.component, p)) continue;
            double w = s.profile ? s.profile[(size_t(k - s.lo[2]) * by + (j - s.lo[1])) * bx + (i - s.lo[0])]
                                 : 1.0;
            if (s.tfsf) w *= sc.eps_inv[g.at(p)];
            st.F[s.component][g.at(p)] += sign * (w * gn);
          }
    }
  }

  // H corrections of the TFSF planes after the H update of step n: H_h += dir S sH profile Einc^n on
  // the scattered-side H plane next to the source plane. With only_R, cells outside R are skipped.
  void add_h_sources(State<T>& st, int n, double sign, bool only_R = false) const {
    for (int q = 0; q < sc.nsrc; ++q) {
      const orc_source& s = sc.src[q];
      if (!s.tfsf) continue;
      const Tfsf& t = tfsf[q];
      const double gn = t.dir * S * t.sH * t.einc[n];
      const int bx = s.hi[0] - s.lo[0], by = s.hi[1] - s.lo[1];
      for (int k = s.lo[2]; k < s.hi[2]; ++k)
        for (int j = s.lo[1]; j < s.hi[1]; ++j)
          for (int i = s.lo[0]; i < s.hi[0]; ++i) {
            int p[3] = {i, j, k};
            p[t.axis] = t.hidx;
            if (only_R && !h_in_R(t.h, p)) continue;
            const double w = s.profile
                                 ? s.profile[(size_t(k - s.lo[2]) * by + (j - s.lo[1])) * bx + (i - s.lo[0])]
                                 : 1.0;
            st.F[3 + t.h][g.at(p)] += sign * (w * gn);
          }
    }
  }

  // Cell-centre values of E_c (mean of 4) and H_c (mean of 2) at cell p; 0 beyond the grid.
  T at_or0(const std::vector<T>& f, const int* p) const {
    for (int d = 0; d < 3; ++d)
      if (p[d] >= g.n[d]) return T(0);
    return f[g.at(p)];
  }
  T e_centre(const std::vector<T>& E, int c, const int* p) const {
    T s = T(0);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        int q[3] = {p[0], p[1], p[2]};
        q[m3(c + 1)] += a;
        q[m3(c + 2)] += b;
        s += at_or0(E, q);
      }
    return 0.25 * s;
  }
  T h_centre(const std::vector<T>& H, int c, const int* p) const {
    int q[3] = {p[0], p[1], p[2]};
    q[c] += 1;
    return 0.5 * (H[g.at(p)] + at_or0(H, q));
  }
  // E^n, kept before the E update of step n when a kind-4 detector needs it
  void keep_prev(const State<T>& st) const {
    if (time_interp)
      for (int c = 0; c < 3; ++c) prevE[c] = st.F[c];
  }

  // Detectors sample E^{n+1} and H^{n+1/2} after step n.
  void sample(const State<T>& st, int n, std::vector<T>& out) const {
    for (int q = 0; q < sc.ndet; ++q) {
      const orc_detector& d = sc.det[q];
      T* o = out.data() + det_offset[q];
      if (d.kind == 0) {
        o[n] = st.F[d.component][g.at(d.lo)];
      } else if (d.kind == 1) {
        size_t m = 0;
        for (int k = d.lo[2]; k < d.hi[2]; ++k)
          for (int j = d.lo[1]; j < d.hi[1]; ++j)
            for (int i = d.lo[0]; i < d.hi[0]; ++i, ++m) {
              const size_t p = g.at(i, j, k);
              o[m] += st.F[0][p] * st.F[0][p] + st.F[1][p] * st.F[1][p] + st.F[2][p] * st.F[2][p];
            }
      } else if (d.kind == 2) {
        const int a1 = m3(d.axis + 1), a2 = m3(d.axis + 2);
        T f = T(0);
        for (int k = d.lo[2]; k < d.hi[2]; ++k)
          for (int j = d.lo[1]; j < d.hi[1]; ++j)
            for (int i = d.lo[0]; i < d.hi[0]; ++i) {
              const size_t p = g.at(i, j, k);
              f += st.F[a1][p] * st.F[3 + a2][p] - st.F[a2][p] * st.F[3 + a1][p];
            }
        o[n] = f;
      } else if (d.kind == 3) {
        size_t m = 0;
        for (int k = d.lo[2]; k < d.hi[2]; ++k)
          for (int j = d.lo[1]; j < d.hi[1]; ++j)
            for (int i = d.lo[0]; i < d.hi[0]; ++i, ++m) {
              const int p[3] = {i, j, k};
              for (int c = 0; c < 3; ++c) {
                const T e = e_centre(st.F[c], c, p);
                o[m] += e * e;
              }
            }
      } else if (d.kind == 4) {
        const int a1 = m3(d.axis + 1), a2 = m3(d.axis + 2);
        T f = T(0);
        for (int k = d.lo[2]; k < d.hi[2]; ++k)
          for (int j = d.lo[1]; j < d.hi[1]; ++j)
            for (int i = d.lo[0]; i < d.hi[0]; ++i) {
              const int p[3] = {i, j, k};
              const T e1 = 0.5 * (e_centre(prevE[a1], a1, p) + e_centre(st.F[a1], a1, p));
              const T e2 = 0.5 * (e_centre(prevE[a2], a2, p) + e_centre(st.F[a2], a2, p));
              f += e1 * h_centre(st.F[3 + a2], a2, p) - e2 * h_centre(st.F[3 + a1], a1, p);
            }
        o[n] = f;
      }
    }
  }

  void step(State<T>& st, int n, std::vector<T>* det) const {
    update_H(st);
    add_h_sources(st, n, +1.0);
    if (det) keep_prev(st);
    update_E(st);
    add_sources(st, n, +1.0);
    if (det) sample(st, n, *det);
  }

  // ---------------------------------------------------------------------------------------------
  // Reverse mode of one step (Sec. 2.2). The adjoint state holds dL/d(state after step n); on return
  // it holds dL/d(state before step n). `fw` is the forward state after step n: only E^{n+1} and
  // H^{n+1/2} at detector cells, and H^{n+1/2} and psi_E at the cells where dL/da is wanted, are
  // read. `gy` holds dL/d(detector outputs).
  // Each forward statement is transposed in turn (scatter form), in reverse order.
  // ---------------------------------------------------------------------------------------------
  // Transposes of e_centre and h_centre: add w times each stencil weight to the stencil points.
  void e_centre_T(std::vector<T>& Eb, int c, const int* p, T w) const {
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        int q[3] = {p[0], p[1], p[2]};
        q[m3(c + 1)] += a;
        q[m3(c + 2)] += b;
        if (q[0] < g.n[0] && q[1] < g.n[1] && q[2] < g.n[2]) Eb[g.at(q)] += 0.25 * w;
      }
  }
  void h_centre_T(std::vector<T>& Hb, int c, const int* p, T w) const {
    Hb[g.at(p)] += 0.5 * w;
    int q[3] = {p[0], p[1], p[2]};
    q[c] += 1;
    if (q[c] < g.n[c]) Hb[g.at(q)] += 0.5 * w;
  }
  // E^n for the kind-4 detectors of step n (the state before the step)
  void set_prev(const State<T>& before) const {
    if (time_interp)
      for (int c = 0; c < 3; ++c) prevE[c] = before.F[c];
  }

  // Detector terms through the state after step n (E^{n+1}, H^{n+1/2}); kind 4 also reads E^n
  // (set_prev) for its H term.
  void inject_detectors(const State<T>& fw, int n, const double* gy, State<T>& ad) const {
    for (int q = 0; q < sc.ndet; ++q) {
      const orc_detector& d = sc.det[q];
      const double* gq = gy + det_offset[q];
      if (d.kind == 0) {
        ad.F[d.component][g.at(d.lo)] += gq[n];
      } else if (d.kind == 1) {
        size_t m = 0;
        for (int k = d.lo[2]; k < d.hi[2]; ++k)
          for (int j = d.lo[1]; j < d.hi[1]; ++j)
            for (int i = d.lo[0]; i < d.hi[0]; ++i, ++m) {
              const size_t p = g.at(i, j, k);
              for (int c = 0; c < 3; ++c) ad.F[c][p] += 2.0 * gq[m] * fw.F[c][p];
            }
      } else if (d.kind == 2) {
        const int a1 = m3(d.axis + 1), a2 = m3(d.axis + 2);
        for (int k = d.lo[2]; k < d.hi[2]; ++k)
          for (int j = d.lo[1]; j < d.hi[1]; ++j)
            for (int i = d.lo[0]; i < d.hi[0]; ++i) {
              const size_t p = g.at(i, j, k);
              ad.F[a1][p] += gq[n] * fw.F[3 + a2][p];
              ad.F[3 + a2][p] += gq[n] * fw.F[a1][p];
              ad.F[a2][p] -= gq[n] * fw.F[3 + a1][p];
              ad.F[3 + a1][p] -= gq[n] * fw.F[a2][p];
            }
      } else if (d.kind == 3) {
        size_t m = 0;
        for (int k = d.lo[2]; k < d.hi[2]; ++k)
          for (int j = d.lo[1]; j < d.hi[1]; ++j)
            for (int i = d.lo[0]; i < d.hi[0]; ++i, ++m) {
              const int p[3] = {i, j, k};
              for (int c = 0; c < 3; ++c) e_centre_T(ad.F[c], c, p, 2.0 * gq[m] * e_centre(fw.F[c], c, p));
            }
      } else if (d.kind == 4) {
        const int a1 = m3(d.axis + 1), a2 = m3(d.axis + 2);
        const T G = T(gq[n]);
        for (int k = d.lo[2]; k < d.hi[2]; ++k)
          for (int j = d.lo[1]; j < d.hi[1]; ++j)
            for (int i = d.lo[0]; i < d.hi[0]; ++i) {
              const int p[3] = {i, j, k};
              const T h1 = h_centre(fw.F[3 + a1], a1, p), h2 = h_centre(fw.F[3 + a2], a2, p);
              const T e1 = 0.5 * (e_centre(prevE[a1], a1, p) + e_centre(fw.F[a1], a1, p));
              const T e2 = 0.5 * (e_centre(prevE[a2], a2, p) + e_centre(fw.F[a2], a2, p));
              // F = e1 h2 - e2 h1, e = (E^n + E^{n+1}) / 2
              e_centre_T(ad.F[a1], a1, p, 0.5 * G * h2);
              e_centre_T(ad.F[a2], a2, p, -0.5 * G * h1);
              h_centre_T(ad.F[3 + a2], a2, p, G * e1);
              h_centre_T(ad.F[3 + a1], a1, p, -G * e2);
            }
      }
    }
  }

  // The kind-4 terms through E^n, added once the adjoint holds dL/d(state before step n).
  void inject_detectors_prev(const State<T>& fw, int n, const double* gy, State<T>& ad) const {
    for (int q = 0; q < sc.ndet; ++q) {
      const orc_detector& d = sc.det[q];
      if (d.kind != 4) continue;
      const int a1 = m3(d.axis + 1), a2 = m3(d.axis + 2);
      const T G = T(gy[det_offset[q] + n]);
      for (int k = d.lo[2]; k < d.hi[2]; ++k)
        for (int j = d.lo[1]; j < d.hi[1]; ++j)
          for (int i = d.lo[0]; i < d.hi[0]; ++i) {
            const int p[3] = {i, j, k};
            e_centre_T(ad.F[a1], a1, p, 0.5 * G * h_centre(fw.F[3 + a2], a2, p));
            e_centre_T(ad.F[a2], a2, p, -0.5 * G * h_centre(fw.F[3 + a1], a1, p));
          }
    }
  }

  // Transpose of update_E. Accumulates dL/da (all cells) from the forward H^{n+1/2} and psi_E.
  void adjoint_E(const State<T>& fw, State<T>& ad, std::vector<T>& dLda) const {
    for (int c = 0; c < 3; ++c) {
      const int c1 = m3(c + 1), c2 = m3(c + 2);
      // serial: the scatter into neighbouring H-adjoint cells is written plainly
      for (int k = 0; k < g.n[2]; ++k)
        for (int j = 0; j < g.n[1]; ++j)
          for (int i = 0; i < g.n[0]; ++i) {
            int p[3] = {i, j, k};
            if (!e_updated(c, p)) continue;
            const size_t q = g.at(p);
            int p1[3] = {i, j, k}; p1[c1] -= 1;
            int p2[3] = {i, j, k}; p2[c2] -= 1;
            const size_t q1 = g.at(p1), q2 = g.at(p2);
            const AxisCoef& A1 = cf[c1];
            const AxisCoef& A2 = cf[c2];
            const double k1 = A1.kappa_int[p[c1]], k2 = A2.kappa_int[p[c2]];
            // forward: E += S a (d1/k1 + s1 - d2/k2 - s2), s = psi after its update
            const T d1 = fw.F[3 + c2][q] - fw.F[3 + c2][q1];
            const T d2 = fw.F[3 + c1][q] - fw.F[3 + c1][q2];
            const T Ebar = ad.F[c][q];
            dLda[q] += S * Ebar * (d1 / k1 + fw.psiE[c][c1][q] - d2 / k2 - fw.psiE[c][c2][q]);
            const T u = S * a[q] * Ebar;
            T& sb1 = ad.psiE[c][c1][q];
            T& sb2 = ad.psiE[c][c2][q];
            sb1 += u;
            sb2 -= u;
            T db1 = u / k1;
            T db2 = -u / k2;
            // forward: s = b s + c d
            db1 += A1.c_int[p[c1]] * sb1;
            sb1 = A1.b_int[p[c1]] * sb1;
            db2 += A2.c_int[p[c2]] * sb2;
            sb2 = A2.b_int[p[c2]] * sb2;
            // forward: d1 = H_{c2}[p] - H_{c2}[p - e_{c1}], d2 = H_{c1}[p] - H_{c1}[p - e_{c2}]
            ad.F[3 + c2][q] += db1;
            ad.F[3 + c2][q1] -= db1;
            ad.F[3 + c1][q] += db2;
            ad.F[3 + c1][q2] -= db2;
          }
    }
  }

  // Transpose of update_H (no parameter dependence: mu = 1).
  void adjoint_H(State<T>& ad) const {
    for (int c = 0; c < 3; ++c) {
      const int c1 = m3(c + 1), c2 = m3(c + 2);
      for (int k = 0; k < g.n[2]; ++k)
        for (int j = 0; j < g.n[1]; ++j)
          for (int i = 0; i < g.n[0]; ++i) {
            int p[3] = {i, j, k};
            const size_t q = g.at(p);
            const AxisCoef& A1 = cf[c1];
            const AxisCoef& A2 = cf[c2];
            // forward: H -= S (d1/k1 + s1 - d2/k2 - s2)
            const T w = -S * ad.F[3 + c][q];
            T& sb1 = ad.psiH[c][c1][q];
            T& sb2 = ad.psiH[c][c2][q];
            sb1 += w;
            sb2 -= w;
            T db1 = w / A1.kappa_half[p[c1]];
            T db2 = -w / A2.kappa_half[p[c2]];
            db1 += A1.c_half[p[c1]] * sb1;
            sb1 = A1.b_half[p[c1]] * sb1;
            db2 += A2.c_half[p[c2]] * sb2;
            sb2 = A2.b_half[p[c2]] * sb2;
            // forward: d1 = E_{c2}[p + e_{c1}] - E_{c2}[p], d2 = E_{c1}[p + e_{c2}] - E_{c1}[p]
            int p1[3] = {i, j, k}; p1[c1] += 1;
            int p2[3] = {i, j, k}; p2[c2] += 1;
            if (p1[c1] < g.n[c1]) ad.F[c2][g.at(p1)] += db1;
            ad.F[c2][q] -= db1;
            if (p2[c2] < g.n[c2]) ad.F[c1][g.at(p2)] += db2;
            ad.F[c1][q] -= db2;
          }
    }
  }

  void adjoint_step(const State<T>& fw, int n, const double* gy, State<T>& ad, std::vector<T>& dLda) const {
    inject_detectors(fw, n, gy, ad);
    // sources add a constant: their transpose is the identity on the adjoint
    adjoint_E(fw, ad, dLda);
    adjoint_H(ad);
    inject_detectors_prev(fw, n, gy, ad);
  }

  // ---------------------------------------------------------------------------------------------
  // Time reversal (Sec. 2.2). R is the set of field components at depth 0 from every PML: along an
  // axis with layers p0, p1 and N cells, integer positions p0 .. min(N - p1, N - 1) and half
  // positions p0 .. N - p1 - 1. Inside R the CPML terms vanish (kappa = 1, c = 0, psi = 0), so the
  // update is invertible there. The E stencils of R read outside R only at the tangential H
  // components on the six planes just outside R; those are recorded after every H update and
  // replayed in reverse.
  // ---------------------------------------------------------------------------------------------
  int int_lo(int d) const { return sc.pml[2 * d]; }
  int int_hi(int d) const { return std::min(g.n[d] - sc.pml[2 * d + 1], g.n[d] - 1); }
  int half_lo(int d) const { return sc.pml[2 * d]; }
  int half_hi(int d) const { return g.n[d] - sc.pml[2 * d + 1] - 1; }

  // (field index, cell) pairs of the face set, in a fixed order.
  std::vector<std::pair<int, size_t>> face_set() const {
    std::vector<std::pair<int, size_t>> fs;
    for (int d = 0; d < 3; ++d) {
      const int e1 = m3(d + 1), e2 = m3(d + 2);
      for (int side = 0; side < 2; ++side) {
        const int p = sc.pml[2 * d + side];
        if (p == 0) continue;
        const int idx = side == 0 ? p - 1 : g.n[d] - p;
        for (int comp : {e1, e2})
          for (int v = int_lo(e2); v <= int_hi(e2); ++v)
            for (int u = int_lo(e1); u <= int_hi(e1); ++u) {
              int q[3];
              q[d] = idx; q[e1] = u; q[e2] = v;
              fs.push_back({3 + comp, g.at(q)});
            }
      }
    }
    return fs;
  }

  void record_faces(const State<T>& st, const std::vector<std::pair<int, size_t>>& fs, std::vector<T>& out) const {
    out.resize(fs.size());
    for (size_t m = 0; m < fs.size(); ++m) out[m] = st.F[fs[m].first][fs[m].second];
  }
  void replay_faces(State<T>& st, const std::vector<std::pair<int, size_t>>& fs, const std::vector<T>& in) const {
    for (size_t m = 0; m < fs.size(); ++m) st.F[fs[m].first][fs[m].second] = in[m];
  }

  // (E^{n+1}, H^{n+1/2}) -> (E^n, H^{n-1/2}) on R; H outside R at the face set must hold step n's record.
  void inverse_step(State<T>& st, int n) const {
    add_sources(st, n, -1.0, true);
    for (int c = 0; c < 3; ++c) {
      const int c1 = m3(c + 1), c2 = m3(c + 2);
      std::vector<T>& E = st.F[c];
      const std::vector<T>& Ha = st.F[3 + c2];
      const std::vector<T>& Hb = st.F[3 + c1];
      int lo[3], hi[3];
      for (int d = 0; d < 3; ++d) {
        lo[d] = (d == c) ? half_lo(d) : int_lo(d);
        hi[d] = (d == c) ? half_hi(d) : int_hi(d);
      }
#pragma omp parallel for
      for (int k = lo[2]; k <= hi[2]; ++k)
        for (int j = lo[1]; j <= hi[1]; ++j)
          for (int i = lo[0]; i <= hi[0]; ++i) {
            int p[3] = {i, j, k};
            if (!e_updated(c, p)) continue;
            const size_t q = g.at(p);
            int p1[3] = {i, j, k}; p1[c1] -= 1;
            int p2[3] = {i, j, k}; p2[c2] -= 1;
            const T d1 = Ha[q] - Ha[g.at(p1)];
            const T d2 = Hb[q] - Hb[g.at(p2)];
            // in R: kappa = 1 and psi = 0, so the forward increment was S a (d1 - d2)
            E[q] -= S * a[q] * (d1 / 1.0 + T(0) - d2 / 1.0 - T(0));
          }
    }
    for (int c = 0; c < 3; ++c) {
      const int c1 = m3(c + 1), c2 = m3(c + 2);
      std::vector<T>& H = st.F[3 + c];
      const std::vector<T>& Ea = st.F[c2];
      const std::vector<T>& Eb = st.F[c1];
      int lo[3], hi[3];
      for (int d = 0; d < 3; ++d) {
        lo[d] = (d == c) ? int_lo(d) : half_lo(d);
        hi[d] = (d == c) ? int_hi(d) : half_hi(d);
      }
#pragma omp parallel for
      for (int k = lo[2]; k <= hi[2]; ++k)
        for (int j = lo[1]; j <= hi[1]; ++j)
          for (int i = lo[0]; i <= hi[0]; ++i) {
            int p[3] = {i, j, k};
            const size_t q = g.at(p);
            int p1[3] = {i, j, k}; p1[c1] += 1;
            int p2[3] = {i, j, k}; p2[c2] += 1;
            const T ea1 = (p1[c1] < g.n[c1]) ? Ea[g.at(p1)] : T(0);
            const T eb2 = (p2[c2] < g.n[c2]) ? Eb[g.at(p2)] : T(0);
            const T d1 = ea1 - Ea[q];
            const T d2 = eb2 - Eb[q];
            H[q] += S * (d1 / 1.0 + T(0) - d2 / 1.0 - T(0));
          }
    }
    add_h_sources(st, n, -1.0, true);
  }

  bool h_in_R(int c, const int* p) const {
    for (int d = 0; d < 3; ++d) {
      const int lo = (d == c) ? int_lo(d) : half_lo(d);
      const int hi = (d == c) ? int_hi(d) : half_hi(d);
      if (p[d] < lo || p[d] > hi) return false;
    }
    return true;
  }

  bool e_in_R(int c, const int* p) const {
    for (int d = 0; d < 3; ++d) {
      const int lo = (d == c) ? half_lo(d) : int_lo(d);
      const int hi = (d == c) ? half_hi(d) : int_hi(d);
      if (p[d] < lo || p[d] > hi) return false;
    }
    return true;
  }

  void load_initial(State<T>& st, const double* init6) const {
    if (!init6) return;
    for (int f = 0; f < 6; ++f)
      for (size_t p = 0; p < g.N; ++p) st.F[f][p] = T(init6[f * g.N + p]);
  }
};

template <class T>
void finish_gradient(const Sim<T>& sim, const std::vector<T>& dLda, double* dL_deps, double* dLda_full) {
  const orc_scene& s = sim.sc;
  if (dL_deps) {
    size_t m = 0;
    for (int k = s.design_lo[2]; k < s.design_hi[2]; ++k)
      for (int j = s.design_lo[1]; j < s.design_hi[1]; ++j)
        for (int i = s.design_lo[0]; i < s.design_hi[0]; ++i, ++m) {
          const size_t p = sim.g.at(i, j, k);
          const double a = s.eps_inv[p];
          dL_deps[m] = -a * a * std::real(dLda[p]);  // a = 1/eps, da/deps = -a^2
        }
  }
  if (dLda_full)
    for (size_t p = 0; p < sim.g.N; ++p) dLda_full[p] = std::real(dLda[p]);
}

}  // namespace

extern "C" {

// Size of the concatenated detector output for nsteps steps.
int64_t orc_detector_total(const orc_scene* s, int32_t nsteps) {
  Sim<double> sim(*s, nsteps);
  return int64_t(sim.det_total);
}

// Number of H values recorded per step by the time-reversal gradient.
int64_t orc_face_count(const orc_scene* s) {
  Sim<double> sim(*s, 1);
  return int64_t(sim.face_set().size());
}

// Forward: nsteps steps from init6 (E^0 then H^{-1/2}, 6*N values, or NULL for zero fields).
// out6 receives E^{nsteps}, H^{nsteps-1/2}; det receives the detector outputs (may be NULL).
int orc_forward(const orc_scene* s, int32_t nsteps, const double* init6, double* out6, double* det) {
  Sim<double> sim(*s, nsteps);
  State<double> st(sim.g.N);
  sim.load_initial(st, init6);
  std::vector<double> d(sim.det_total, 0.0);
  for (int n = 0; n < nsteps; ++n) sim.step(st, n, &d);
  if (out6)
    for (int f = 0; f < 6; ++f) std::memcpy(out6 + f * sim.g.N, st.F[f].data(), sim.g.N * sizeof(double));
  if (det) std::memcpy(det, d.data(), d.size() * sizeof(double));
  return 0;
}

// Forward nsteps with face recording, then nsteps inverse steps (Sec. 2.2 time reversal).
// out_fwd6: state after the forward; out_back6: state after the reversal (meaningful on R only).
int orc_roundtrip(const orc_scene* s, int32_t nsteps, const double* init6, double* out_fwd6, double* out_back6) {
  Sim<double> sim(*s, nsteps);
  State<double> st(sim.g.N);
  sim.load_initial(st, init6);
  const auto fs = sim.face_set();
  std::vector<std::vector<double>> rec(nsteps);
  for (int n = 0; n < nsteps; ++n) {
    sim.update_H(st);
    sim.add_h_sources(st, n, +1.0);
    sim.record_faces(st, fs, rec[n]);
    sim.update_E(st);
    sim.add_sources(st, n, +1.0);
  }
  if (out_fwd6)
    for (int f = 0; f < 6; ++f) std::memcpy(out_fwd6 + f * sim.g.N, st.F[f].data(), sim.g.N * sizeof(double));
  for (int n = nsteps - 1; n >= 0; --n) {
    sim.replay_faces(st, fs, rec[n]);
    sim.inverse_step(st, n);
  }
  if (out_back6)
    for (int f = 0; f < 6; ++f) std::memcpy(out_back6 + f * sim.g.N, st.F[f].data(), sim.g.N * sizeof(double));
  return 0;
}

// Reverse-mode gradient of L = sum(dL_ddet * detectors) with respect to eps on the design box, for
// the forward from init6 (E^0 then H^{-1/2}, 6*N values, or NULL for zero fields).
//   method 0: store every state (tiny grids only)
//   method 1: full-state checkpoint every `interval` steps, recompute each segment
//   method 2: time reversal with face record and replay
// dL_deps: design-box-shaped output (x fastest). dLda_full: optional N-sized dL/da (methods 0, 1).
// det: optional detector outputs of the forward pass.
int orc_gradient_from(const orc_scene* s, int32_t nsteps, const double* init6, const double* dL_ddet,
                      int32_t method, int32_t interval, double* dL_deps, double* dLda_full, double* det) {
  Sim<double> sim(*s, nsteps);
  const size_t N = sim.g.N;
  std::vector<double> dLda(N, 0.0);
  std::vector<double> d(sim.det_total, 0.0);
  State<double> ad(N);
  if (method == 0) {
    std::vector<State<double>> traj(nsteps + 1, State<double>(0));
    traj[0].resize(N);
    sim.load_initial(traj[0], init6);
    for (int n = 0; n < nsteps; ++n) {
      traj[n + 1] = traj[n];
      sim.step(traj[n + 1], n, &d);
    }
    for (int n = nsteps - 1; n >= 0; --n) {
      sim.set_prev(traj[n]);
      sim.adjoint_step(traj[n + 1], n, dL_ddet, ad, dLda);
    }
  } else if (method == 1) {
    if (interval < 1) return -1;
    std::vector<State<double>> ckpt;
    State<double> st(N);
    sim.load_initial(st, init6);
    for (int n = 0; n < nsteps; ++n) {
      if (n % interval == 0) ckpt.push_back(st);
      sim.step(st, n, &d);
    }
    for (int seg = int(ckpt.size()) - 1; seg >= 0; --seg) {
      const int n0 = seg * interval, n1 = std::min(nsteps, n0 + interval);
      std::vector<State<double>> traj;
      traj.push_back(ckpt[seg]);
      for (int n = n0; n < n1; ++n) {
        traj.push_back(traj.back());
        sim.step(traj.back(), n, nullptr);
      }
      for (int n = n1 - 1; n >= n0; --n) {
        sim.set_prev(traj[n - n0]);
        sim.adjoint_step(traj[n - n0 + 1], n, dL_ddet, ad, dLda);
      }
    }
  } else if (method == 2) {
    State<double> st(N);
    sim.load_initial(st, init6);
    const auto fs = sim.face_set();
    std::vector<std::vector<double>> rec(nsteps);
    for (int n = 0; n < nsteps; ++n) {
      sim.update_H(st);
      sim.add_h_sources(st, n, +1.0);
      sim.record_faces(st, fs, rec[n]);
      sim.keep_prev(st);
      sim.update_E(st);
      sim.add_sources(st, n, +1.0);
      sim.sample(st, n, d);
    }
    for (int n = nsteps - 1; n >= 0; --n) {
      // st holds E^{n+1} and H^{n+1/2} on R; psi_E is zero on R
      sim.replay_faces(st, fs, rec[n]);
      if (sim.time_interp) {  // E^n on R, by one inverse step on a copy
        State<double> before = st;
        sim.inverse_step(before, n);
        sim.set_prev(before);
      }
      sim.adjoint_step(st, n, dL_ddet, ad, dLda);
      sim.inverse_step(st, n);
    }
  } else {
    return -1;
  }
  finish_gradient(sim, dLda, dL_deps, (method == 2) ? nullptr : dLda_full);
  if (det) std::memcpy(det, d.data(), d.size() * sizeof(double));
  return 0;
}

int orc_gradient(const orc_scene* s, int32_t nsteps, const double* dL_ddet, int32_t method, int32_t interval,
                 double* dL_deps, double* dLda_full, double* det) {
  return orc_gradient_from(s, nsteps, nullptr, dL_ddet, method, interval, dL_deps, dLda_full, det);
}

// Complex-step derivative dL/deps at each listed voxel: eps_v -> eps_v + i h, one forward per voxel,
// dL/deps_v = Im(L) / h with L = sum(dL_ddet * detectors).
int orc_complex_step(const orc_scene* s, int32_t nsteps, const double* dL_ddet, int32_t nvox, const int32_t* vox,
                     double h, double* out) {
  for (int v = 0; v < nvox; ++v) {
    Sim<cplx> sim(*s, nsteps);
    const size_t p = sim.g.at(vox[3 * v], vox[3 * v + 1], vox[3 * v + 2]);
    const double eps = 1.0 / s->eps_inv[p];
    sim.a[p] = 1.0 / cplx(eps, h);
    State<cplx> st(sim.g.N);
    std::vector<cplx> d(sim.det_total, cplx(0));
    for (int n = 0; n < nsteps; ++n) sim.step(st, n, &d);
    cplx L = 0;
    for (size_t m = 0; m < d.size(); ++m) L += dL_ddet[m] * d[m];
    out[v] = std::imag(L) / h;
  }
  return 0;
}

// CPML coefficient tables of one axis (for inspection): six arrays of n[axis] values each, in the
// order b_int, c_int, kappa_int, b_half, c_half, kappa_half.
int orc_cpml_tables(const orc_scene* s, int32_t axis, double* out) {
  const auto cf = make_coefs(*s);
  const AxisCoef& a = cf[axis];
  const int N = s->n[axis];
  const std::vector<double>* v[6] = {&a.b_int, &a.c_int, &a.kappa_int, &a.b_half, &a.c_half, &a.kappa_half};
  for (int t = 0; t < 6; ++t) std::memcpy(out + t * N, v[t]->data(), N * sizeof(double));
  return 0;
}

// Detector outputs of one step sampled from given fields (for inspection): prev6 supplies E^n (its
// first three arrays; may be NULL for E^n = E^{n+1}), state6 the fields after the step (E^{n+1},
// H^{n+1/2}); out receives orc_detector_total(s, 1) values.
int orc_sample(const orc_scene* s, const double* prev6, const double* state6, double* out) {
  Sim<double> sim(*s, 1);
  State<double> st(sim.g.N);
  sim.load_initial(st, state6);
  for (int c = 0; c < 3; ++c) {
    sim.prevE[c] = st.F[c];
    if (prev6) std::memcpy(sim.prevE[c].data(), prev6 + c * sim.g.N, sim.g.N * sizeof(double));
  }
  std::vector<double> d(sim.det_total, 0.0);
  sim.sample(st, 0, d);
  std::memcpy(out, d.data(), d.size() * sizeof(double));
  return 0;
}

// Source waveform g(s) of source q at fractional step s (for inspection).
double orc_waveform(const orc_scene* s, int32_t q, double step) { return waveform(s->src[q], s->courant, step); }

}  // extern "C"
