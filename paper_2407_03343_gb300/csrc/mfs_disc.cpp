// Host discretisation of P equal spheres for the image-enhanced MFS.
//
// Sec. 2.1  basic grids: N proxy Stokeslets on radius R_p a, M0 collocation nodes on the
//           surface.  Quasi-uniform Fibonacci grids stand in for the spherical designs the
//           paper uses (its own alternative): cos(theta_j) = 1 - (2j - 1)/n,
//           phi_j = 2 pi j / Phi mod 2 pi, j = 1..n, in the global frame, so every
//           sphere without contacts has the same self block.
// Sec. 2.3  contacts (gap delta = |c_k - c_k'|/a - 2), accumulation radius eq. Racc,
//           image nodes t_j of eq. tj on the line of eq. line_points.
// Sec. 5.1  n_im from eq. image_est (capped at nim_max), two collocation caps per contact
//           per sphere with M_cap = alpha * 3 n_im nodes (eq. colloc_nbr) placed by
//           eq. thetacap read as cos(theta_j) = 1 - j (1 - cos beta)/M_cap (half-angle beta),
//           area weights 4 pi a^2 / M0 and 2 pi a^2 (1 - cos beta) / M_cap.
// Contact frame about the unit axis e: h = e_z if |e_z| <= 0.9 else e_x,
// e1 = normalise(h - (h.e) e), e2 = e x e1.  Partners are visited in ascending index.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "mfs_internal.h"

namespace mfs {
namespace {

const double kPi = 3.14159265358979323846;
const double kGolden = 1.6180339887498948482;

void fib_direction(int j, int n, double cos_t, double* d) {
  (void)n;
  double sin_t = std::sqrt(std::max(0.0, 1.0 - cos_t * cos_t));
  double phi = std::fmod(2.0 * kPi * j / kGolden, 2.0 * kPi);
  d[0] = sin_t * std::cos(phi);
  d[1] = sin_t * std::sin(phi);
  d[2] = cos_t;
}

// eq. Racc for a unit sphere.
double racc(double delta) { return 1.0 + 0.5 * delta - std::sqrt(delta + 0.25 * delta * delta); }

int image_count(double delta, const mfs_params& p) {
  if (delta >= p.nim_cut) return 0;
  if (p.nim_fixed >= 0) return p.nim_fixed;
  double v = std::ceil(-p.nim_a * std::log10(delta) - p.nim_b);
  if (v < p.nim_min) v = p.nim_min;
  if (v < 0) v = 0;
  if (v > p.nim_max) v = p.nim_max;
  return (int)v;
}

void perp_frame(const double* e, double* e1, double* e2) {
  double h[3] = {0.0, 0.0, 1.0};
  if (std::fabs(e[2]) > 0.9) { h[0] = 1.0; h[2] = 0.0; }
  double hd = h[0] * e[0] + h[1] * e[1] + h[2] * e[2];
  for (int i = 0; i < 3; ++i) e1[i] = h[i] - hd * e[i];
  double nn = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  for (int i = 0; i < 3; ++i) e1[i] /= nn;
  e2[0] = e[1] * e1[2] - e[2] * e1[1];
  e2[1] = e[2] * e1[0] - e[0] * e1[2];
  e2[2] = e[0] * e1[1] - e[1] * e1[0];
}

}  // namespace

void fibonacci_sphere(int n, double r, std::vector<double>& out) {
  out.assign(3 * (size_t)n, 0.0);
  for (int j = 1; j <= n; ++j) {
    double d[3];
    fib_direction(j, n, 1.0 - (2.0 * j - 1.0) / n, d);
    for (int q = 0; q < 3; ++q) out[3 * (size_t)(j - 1) + q] = r * d[q];
  }
}

mfs_status build_discretisation(const double* centres, int P, double a, const mfs_params& p,
                                HostDisc& out, std::string& err) {
  if (P <= 0 || p.n_proxy <= 0 || p.m_basic <= 0 || !(a > 0) || !(p.r_proxy > 0) || p.r_proxy >= 1.0 ||
      p.alpha1 < 0 || p.alpha2 < 0 || !(p.visc > 0) || p.nim_max < 0 || p.nim_min < 0 || p.nim_min > p.nim_max) {
    err = "invalid discretisation parameters";
    return MFS_ERR_ARG;
  }
  if (p.far_dist < 0 || (p.far_dist > 0 && (p.far_n_eq < 4 || !(p.far_r_eq > 0) || !(p.far_r_chk > p.far_r_eq) ||
                                             p.far_dist < p.far_r_chk + 1.0 || !(p.far_eps > 0) || p.far_eps >= 1))) {
    err = "invalid far-field parameters (need n_eq >= 4, 0 < r_eq < r_chk, far_dist >= r_chk + 1, 0 < eps < 1)";
    return MFS_ERR_ARG;
  }
  HostDisc d;
  d.P = P;
  d.a = a;
  d.prm = p;
  d.centres.assign(centres, centres + 3 * (size_t)P);

  // contacts, all pairs k < kp
  std::vector<std::vector<std::pair<int, int>>> per(P);  // (partner, contact index)
  for (int k = 0; k < P; ++k) {
    for (int kp = k + 1; kp < P; ++kp) {
      double dx = centres[3 * kp] - centres[3 * k], dy = centres[3 * kp + 1] - centres[3 * k + 1],
             dz = centres[3 * kp + 2] - centres[3 * k + 2];
      double dist = std::sqrt(dx * dx + dy * dy + dz * dz);
      double delta = dist / a - 2.0;
      if (!(delta > 0.0)) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "spheres %d and %d overlap or touch (gap %.3e radii)", k, kp, delta);
        err = buf;
        return MFS_ERR_GEOMETRY;
      }
      int n = image_count(delta, p);
      if (n > 0) {
        int ci = (int)d.contacts.size();
        d.contacts.push_back({k, kp, delta, n});
        per[k].push_back({kp, ci});
        per[kp].push_back({k, ci});
      }
    }
  }
  for (auto& v : per) std::sort(v.begin(), v.end());

  const int N = p.n_proxy, M0 = p.m_basic;
  d.proxy_rel.resize(3 * (size_t)N);
  for (int j = 1; j <= N; ++j) {
    double dir[3];
    fib_direction(j, N, 1.0 - (2.0 * j - 1.0) / N, dir);
    for (int c = 0; c < 3; ++c) d.proxy_rel[3 * (j - 1) + c] = a * p.r_proxy * dir[c];
  }
  std::vector<double> basic(3 * (size_t)M0);
  for (int j = 1; j <= M0; ++j) {
    double dir[3];
    fib_direction(j, M0, 1.0 - (2.0 * j - 1.0) / M0, dir);
    for (int c = 0; c < 3; ++c) basic[3 * (j - 1) + c] = dir[c];
  }
  const double w_basic = 4.0 * kPi * a * a / M0;
  const double t0 = p.r_proxy * (1.0 + p.delta_offset);

  d.colloc_off.assign(P + 1, 0);
  d.img_off.assign(P + 1, 0);
  d.unk_off.assign(P + 1, 0);
  for (int k = 0; k < P; ++k) {
    const double* ck = &centres[3 * k];
    for (int j = 0; j < M0; ++j) {
      for (int c = 0; c < 3; ++c) d.colloc.push_back(ck[c] + a * basic[3 * j + c]);
      d.weight.push_back(w_basic);
      d.owner.push_back(k);
    }
    int n_img_k = 0;
    for (auto& pc : per[k]) {
      const Contact& ct = d.contacts[pc.second];
      int kp = pc.first;
      double e[3] = {centres[3 * kp] - ck[0], centres[3 * kp + 1] - ck[1], centres[3 * kp + 2] - ck[2]};
      double ne = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
      for (int c = 0; c < 3; ++c) e[c] /= ne;
      double e1[3], e2[3];
      perp_frame(e, e1, e2);
      // image nodes, eq. tj
      double ra = racc(ct.delta);
      for (int j = 1; j <= ct.nim; ++j) {
        double t = t0 + (ra - t0) * std::cos((j - 1.0) / (2.0 * ct.nim) * kPi);
        for (int c = 0; c < 3; ++c) d.image.push_back(ck[c] + a * t * e[c]);
        d.img_owner.push_back(k);
      }
      n_img_k += ct.nim;
      // two caps, eq. colloc_nbr / eq. thetacap
      const int alphas[2] = {p.alpha1, p.alpha2};
      const double betas[2] = {p.beta1, p.beta2};
      for (int cap = 0; cap < 2; ++cap) {
        int m = alphas[cap] * 3 * ct.nim;
        double wc = 2.0 * kPi * a * a * (1.0 - std::cos(betas[cap])) / m;
        for (int j = 1; j <= m; ++j) {
          double cos_t = 1.0 - j * (1.0 - std::cos(betas[cap])) / m;
          double loc[3];
          fib_direction(j, m, cos_t, loc);
          for (int c = 0; c < 3; ++c)
            d.colloc.push_back(ck[c] + a * (loc[0] * e1[c] + loc[1] * e2[c] + loc[2] * e[c]));
          d.weight.push_back(wc);
          d.owner.push_back(k);
        }
      }
    }
    d.colloc_off[k + 1] = (int)d.weight.size();
    d.img_off[k + 1] = d.img_off[k] + n_img_k;
    d.unk_off[k + 1] = d.unk_off[k] + 3LL * N + 9LL * n_img_k;
  }

  // one-body factors: all contact-free spheres share the basic block (global-frame grids)
  d.factor_id.assign(P, -1);
  int shared = -1;
  for (int k = 0; k < P; ++k) {
    if (per[k].empty()) {
      if (shared < 0) {
        shared = (int)d.factor_rep.size();
        d.factor_rep.push_back(k);
      }
      d.factor_id[k] = shared;
    } else {
      d.factor_id[k] = (int)d.factor_rep.size();
      d.factor_rep.push_back(k);
    }
  }
  out = std::move(d);
  return MFS_OK;
}

}  // namespace mfs
