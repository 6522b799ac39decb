// Host-side setup: quadrature, nodal reference operators, mesh connectivity.
#include "dg_host.h"

#include <algorithm>
#include <cmath>
#include <unordered_map>

namespace dgswe {

namespace {

// Cyclic Jacobi eigenvalue iteration for a small dense symmetric matrix.
void sym_eigenvalues(int n, std::vector<double> A, std::vector<double>& ev) {
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    if (off < 1e-34) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A R
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- R^T A
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
      }
    }
  }
  ev.resize(n);
  for (int i = 0; i < n; ++i) ev[i] = A[i * n + i];
  std::sort(ev.begin(), ev.end());
}

bool invert(int n, const std::vector<double>& A, std::vector<double>& Ainv) {
  std::vector<double> a(A);
  Ainv.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) Ainv[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[r * n + c]) > std::fabs(a[piv * n + c])) piv = r;
    if (std::fabs(a[piv * n + c]) < 1e-300) return false;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(a[c * n + k], a[piv * n + k]);
        std::swap(Ainv[c * n + k], Ainv[piv * n + k]);
      }
    double d = 1.0 / a[c * n + c];
    for (int k = 0; k < n; ++k) {
      a[c * n + k] *= d;
      Ainv[c * n + k] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = a[r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[r * n + k] -= f * a[c * n + k];
        Ainv[r * n + k] -= f * Ainv[c * n + k];
      }
    }
  }
  return true;
}

// Monomial exponents (a, b) of total degree <= p (b = 0 in 1D).
std::vector<std::pair<int, int>> monomials(int dim, int p) {
  std::vector<std::pair<int, int>> m;
  if (dim == 1) {
    for (int a = 0; a <= p; ++a) m.push_back({a, 0});
  } else {
    for (int t = 0; t <= p; ++t)
      for (int b = 0; b <= t; ++b) m.push_back({t - b, b});
  }
  return m;
}

double ipow(double x, int k) {
  double r = 1.0;
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}

}  // namespace

void gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w) {
  // Monic three-term recurrence p_{k+1} = (x - al_k) p_k - be_k p_{k-1}.
  std::vector<double> al(n), be(n + 1, 0.0);
  for (int k = 0; k < n; ++k) {
    double s = 2.0 * k + a + b;
    al[k] = (k == 0) ? (b - a) / (a + b + 2.0) : (b * b - a * a) / (s * (s + 2.0));
  }
  for (int k = 1; k <= n; ++k) {
    double s = 2.0 * k + a + b;
    if (k == 1)
      be[k] = 4.0 * (1.0 + a) * (1.0 + b) / ((2.0 + a + b) * (2.0 + a + b) * (3.0 + a + b));
    else
      be[k] = 4.0 * k * (k + a) * (k + b) * (k + a + b) / (s * s * (s + 1.0) * (s - 1.0));
  }
  std::vector<double> T(n * n, 0.0);
  for (int k = 0; k < n; ++k) {
    T[k * n + k] = al[k];
    if (k + 1 < n) T[k * n + k + 1] = T[(k + 1) * n + k] = std::sqrt(be[k + 1]);
  }
  sym_eigenvalues(n, T, x);
  double mu0 = std::pow(2.0, a + b + 1.0) * std::tgamma(a + 1.0) * std::tgamma(b + 1.0) /
               std::tgamma(a + b + 2.0);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    // Newton polish on the monic p_n, then Christoffel weight.
    for (int it = 0; it < 3; ++it) {
      double p0 = 1.0, p1 = x[i] - al[0], d0 = 0.0, d1 = 1.0;
      if (n == 1) { p1 = x[i] - al[0]; d1 = 1.0; }
      for (int k = 1; k < n; ++k) {
        double p2 = (x[i] - al[k]) * p1 - be[k] * p0;
        double d2 = p1 + (x[i] - al[k]) * d1 - be[k] * d0;
        p0 = p1; p1 = p2; d0 = d1; d1 = d2;
      }
      if (d1 != 0.0) x[i] -= p1 / d1;
    }
    double sum = 1.0 / mu0, pk_m1 = 0.0, pk = 1.0, norm = mu0;
    for (int k = 0; k + 1 < n; ++k) {
      double pn = (x[i] - al[k]) * pk - be[k] * pk_m1;
      norm *= be[k + 1];
      sum += pn * pn / norm;
      pk_m1 = pk; pk = pn;
    }
    w[i] = 1.0 / sum;
  }
}

bool build_refops(int dim, int p, RefOps& o, std::string& err) {
  if (dim < 1 || dim > 2 || p < 1 || p > 3) {
    err = "supported: dim in {1,2}, order in {1,2,3}";
    return false;
  }
  o.dim = dim;
  o.p = p;
  o.nf = dim + 1;
  o.Np = dim == 1 ? p + 1 : (p + 1) * (p + 2) / 2;
  o.Nfp = dim == 1 ? 1 : p + 1;
  const int nv = (3 * p + 1) / 2;       // ceil(3p/2)
  const int nfq = (3 * p + 2) / 2;      // ceil((3p+1)/2)
  const int Np = o.Np;
  // nodes
  o.rnodes.clear();
  if (dim == 1) {
    for (int i = 0; i <= p; ++i) o.rnodes.push_back(-1.0 + 2.0 * i / p);
  } else {
    for (int j = 0; j <= p; ++j)
      for (int i = 0; i <= p - j; ++i) {
        o.rnodes.push_back(-1.0 + 2.0 * i / p);
        o.rnodes.push_back(-1.0 + 2.0 * j / p);
      }
  }
  // quadrature
  std::vector<double> ga, wa;
  gauss_jacobi(nv, 0.0, 0.0, ga, wa);
  o.rq.clear();
  o.wq.clear();
  if (dim == 1) {
    o.rq = ga;
    o.wq = wa;
  } else {
    std::vector<double> gb, wb;
    gauss_jacobi(nv, 1.0, 0.0, gb, wb);
    for (int i = 0; i < nv; ++i)
      for (int j = 0; j < nv; ++j) {
        o.rq.push_back(0.5 * (1.0 + ga[i]) * (1.0 - gb[j]) - 1.0);
        o.rq.push_back(gb[j]);
        o.wq.push_back(0.5 * wa[i] * wb[j]);
      }
  }
  o.Nq = (int)o.wq.size();
  // Lagrange basis through a monomial Vandermonde matrix
  auto mono = monomials(dim, p);
  std::vector<double> V(Np * Np), C;
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) {
      double r = o.rnodes[i * dim], s = dim == 2 ? o.rnodes[i * dim + 1] : 0.0;
      V[i * Np + j] = ipow(r, mono[j].first) * ipow(s, mono[j].second);
    }
  if (!invert(Np, V, C)) {
    err = "singular Vandermonde matrix";
    return false;
  }
  auto lagr = [&](double r, double s, double* l, double* lr, double* ls) {
    for (int a = 0; a < Np; ++a) {
      double v = 0, vr = 0, vs = 0;
      for (int j = 0; j < Np; ++j) {
        int ea = mono[j].first, eb = mono[j].second;
        double c = C[j * Np + a];
        v += c * ipow(r, ea) * ipow(s, eb);
        if (ea > 0) vr += c * ea * ipow(r, ea - 1) * ipow(s, eb);
        if (eb > 0) vs += c * eb * ipow(r, ea) * ipow(s, eb - 1);
      }
      l[a] = v;
      lr[a] = vr;
      ls[a] = vs;
    }
  };
  o.Vq.assign(o.Nq * Np, 0);
  o.Drq.assign(o.Nq * Np, 0);
  o.Dsq.assign(o.Nq * Np, 0);
  for (int q = 0; q < o.Nq; ++q) {
    double r = o.rq[q * dim], s = dim == 2 ? o.rq[q * dim + 1] : 0.0;
    lagr(r, s, &o.Vq[q * Np], &o.Drq[q * Np], &o.Dsq[q * Np]);
  }
  o.Dr.assign(Np * Np, 0);
  o.Ds.assign(Np * Np, 0);
  std::vector<double> l(Np), lr(Np), ls(Np);
  for (int a = 0; a < Np; ++a) {
    double r = o.rnodes[a * dim], s = dim == 2 ? o.rnodes[a * dim + 1] : 0.0;
    lagr(r, s, l.data(), lr.data(), ls.data());
    for (int b = 0; b < Np; ++b) {
      o.Dr[a * Np + b] = lr[b];
      o.Ds[a * Np + b] = ls[b];
    }
  }
  o.M.assign(Np * Np, 0);
  o.wint.assign(Np, 0);
  for (int q = 0; q < o.Nq; ++q)
    for (int a = 0; a < Np; ++a) {
      o.wint[a] += o.wq[q] * o.Vq[q * Np + a];
      for (int b = 0; b < Np; ++b) o.M[a * Np + b] += o.wq[q] * o.Vq[q * Np + a] * o.Vq[q * Np + b];
    }
  if (!invert(Np, o.M, o.Minv)) {
    err = "singular mass matrix";
    return false;
  }
  // faces
  o.fmask.assign(o.nf * o.Nfp, 0);
  for (int f = 0; f < o.nf; ++f)
    for (int k = 0; k < o.Nfp; ++k) o.fmask[f * o.Nfp + k] = face_node(dim, p, f, k);
  if (dim == 1) {
    o.Nfq = 1;
    o.tf = {0.0};
    o.wf = {1.0};
    o.Lf = {1.0};
  } else {
    gauss_jacobi(nfq, 0.0, 0.0, o.tf, o.wf);
    o.Nfq = nfq;
    o.Lf.assign(nfq * o.Nfp, 0);
    for (int m = 0; m < nfq; ++m)
      for (int k = 0; k <= p; ++k) {
        double v = 1.0, tk = -1.0 + 2.0 * k / p;
        for (int j = 0; j <= p; ++j)
          if (j != k) v *= (o.tf[m] - (-1.0 + 2.0 * j / p)) / (tk - (-1.0 + 2.0 * j / p));
        o.Lf[m * o.Nfp + k] = v;
      }
  }
  // LIFT = M^-1 * face mass (face nodes)
  std::vector<double> M1(o.Nfp * o.Nfp, 0.0);
  for (int m = 0; m < o.Nfq; ++m)
    for (int k = 0; k < o.Nfp; ++k)
      for (int j = 0; j < o.Nfp; ++j) M1[k * o.Nfp + j] += o.wf[m] * o.Lf[m * o.Nfp + k] * o.Lf[m * o.Nfp + j];
  const int nl = o.nf * o.Nfp;
  o.LIFT.assign(Np * nl, 0.0);
  for (int a = 0; a < Np; ++a)
    for (int f = 0; f < o.nf; ++f)
      for (int j = 0; j < o.Nfp; ++j) {
        double v = 0;
        for (int k = 0; k < o.Nfp; ++k) v += o.Minv[a * Np + o.fmask[f * o.Nfp + k]] * M1[k * o.Nfp + j];
        o.LIFT[a * nl + f * o.Nfp + j] = v;
      }
  return true;
}

bool build_mesh(int dim, int64_t nvtx, const double* X, int64_t K, const int32_t* etov,
                const int8_t* face_bc, int n_bc, const RefOps& ops, MeshData& m,
                std::string& err) {
  const int nf = dim + 1, nvpe = dim + 1, Np = ops.Np;
  m.dim = dim;
  m.nf = nf;
  m.K = K;
  m.geo.assign(kGeoRows * K, 0.0);
  m.nbr.assign(nf * K, 0);
  m.nbrf.assign(nf * K, 0);
  m.fid.assign(nf * K, 0);
  m.fn.assign((size_t)nf * dim * K, 0.0);
  m.fsj.assign(nf * K, 0.0);
  m.node_xyz.assign((size_t)K * Np * dim, 0.0);
  for (int64_t e = 0; e < K; ++e)
    for (int v = 0; v < nvpe; ++v) {
      int32_t id = etov[e * nvpe + v];
      if (id < 0 || id >= nvtx) {
        err = "element vertex index out of range";
        return false;
      }
    }
  // geometry
  for (int64_t e = 0; e < K; ++e) {
    const int32_t* ev = etov + e * nvpe;
    if (dim == 1) {
      double x0 = X[ev[0]], x1 = X[ev[1]];
      double J = 0.5 * (x1 - x0);
      if (!(J > 0)) {
        err = "interval elements must have x1 > x0";
        return false;
      }
      m.geo[0 * K + e] = 1.0 / J;
      m.geo[4 * K + e] = J;
      m.geo[5 * K + e] = 2.0 * J;
      m.geo[6 * K + e] = 1.0 / J;
      m.fn[(0 * dim + 0) * K + e] = -1.0;
      m.fn[(1 * dim + 0) * K + e] = 1.0;
      m.fsj[0 * K + e] = 1.0;
      m.fsj[1 * K + e] = 1.0;
      for (int a = 0; a < Np; ++a) {
        double lam = 0.5 * (1.0 + ops.rnodes[a]);
        m.node_xyz[(e * Np + a)] = x0 * (1.0 - lam) + x1 * lam;
      }
    } else {
      double x0 = X[ev[0] * 2], y0 = X[ev[0] * 2 + 1];
      double x1 = X[ev[1] * 2], y1 = X[ev[1] * 2 + 1];
      double x2 = X[ev[2] * 2], y2 = X[ev[2] * 2 + 1];
      double xr = 0.5 * (x1 - x0), yr = 0.5 * (y1 - y0);
      double xs = 0.5 * (x2 - x0), ys = 0.5 * (y2 - y0);
      double J = xr * ys - xs * yr;
      if (!(J > 0)) {
        err = "triangles must be counter-clockwise with positive area";
        return false;
      }
      m.geo[0 * K + e] = ys / J;   // dr/dx
      m.geo[1 * K + e] = -xs / J;  // dr/dy
      m.geo[2 * K + e] = -yr / J;  // ds/dx
      m.geo[3 * K + e] = xr / J;   // ds/dy
      m.geo[4 * K + e] = J;
      double px[3] = {x0, x1, x2}, py[3] = {y0, y1, y2};
      double perim = 0.0;
      for (int f = 0; f < 3; ++f) {
        double tx = px[(f + 1) % 3] - px[f], ty = py[(f + 1) % 3] - py[f];
        double len = std::sqrt(tx * tx + ty * ty);
        perim += len;
        m.fn[(f * 2 + 0) * K + e] = ty / len;
        m.fn[(f * 2 + 1) * K + e] = -tx / len;
        m.fsj[f * K + e] = 0.5 * len;
      }
      m.geo[5 * K + e] = 4.0 * (2.0 * J) / perim;  // twice the inradius
      m.geo[6 * K + e] = 1.0 / J;
      for (int a = 0; a < Np; ++a) {
        double l1 = 0.5 * (1.0 + ops.rnodes[a * 2]), l2 = 0.5 * (1.0 + ops.rnodes[a * 2 + 1]);
        double l0 = 1.0 - l1 - l2;
        m.node_xyz[(e * Np + a) * 2 + 0] = l0 * x0 + l1 * x1 + l2 * x2;
        m.node_xyz[(e * Np + a) * 2 + 1] = l0 * y0 + l1 * y1 + l2 * y2;
      }
    }
  }
  // connectivity
  std::unordered_map<uint64_t, int64_t> open;  // key -> e*nf+f
  open.reserve((size_t)K * nf);
  m.face_e1.clear();
  m.face_e2.clear();
  m.face_f1.clear();
  m.face_f2.clear();
  auto key_of = [&](int64_t e, int f) -> uint64_t {
    const int32_t* ev = etov + e * nvpe;
    if (dim == 1) return (uint64_t)(uint32_t)ev[f];
    uint32_t a = (uint32_t)ev[f], b = (uint32_t)ev[(f + 1) % 3];
    if (a > b) std::swap(a, b);
    return ((uint64_t)a << 32) | b;
  };
  for (int64_t e = 0; e < K; ++e) {
    for (int f = 0; f < nf; ++f) {
      uint64_t k = key_of(e, f);
      auto it = open.find(k);
      if (it == open.end()) {
        open.emplace(k, e * nf + f);
        continue;
      }
      int64_t e1 = it->second / nf;
      int f1 = (int)(it->second % nf);
      open.erase(it);
      if (dim == 1 && f1 == f) {
        err = "1D elements overlap";
        return false;
      }
      if (dim == 2) {
        const int32_t* a = etov + e1 * 3;
        const int32_t* b = etov + e * 3;
        if (!(a[f1] == b[(f + 1) % 3] && a[(f1 + 1) % 3] == b[f])) {
          err = "adjacent triangles must have opposite edge orientation (all counter-clockwise)";
          return false;
        }
      }
      int32_t id = (int32_t)m.face_e1.size();
      m.face_e1.push_back((int32_t)e1);
      m.face_f1.push_back((int8_t)f1);
      m.face_e2.push_back((int32_t)e);
      m.face_f2.push_back((int8_t)f);
      m.nbr[f1 * K + e1] = (int32_t)e;
      m.nbrf[f1 * K + e1] = (int8_t)f;
      m.fid[f1 * K + e1] = id;
      m.nbr[f * K + e] = (int32_t)e1;
      m.nbrf[f * K + e] = (int8_t)f1;
      m.fid[f * K + e] = id | (int32_t)0x80000000;
    }
  }
  // remaining faces are boundary faces
  std::vector<int64_t> bnd;
  bnd.reserve(open.size());
  for (auto& kv : open) bnd.push_back(kv.second);
  std::sort(bnd.begin(), bnd.end());
  for (int64_t ef : bnd) {
    int64_t e = ef / nf;
    int f = (int)(ef % nf);
    int bc = face_bc ? (int)face_bc[e * nf + f] : 0;
    if (bc < 0 || bc >= n_bc) {
      err = "boundary face tag out of range of the boundary-condition table";
      return false;
    }
    int32_t id = (int32_t)m.face_e1.size();
    m.face_e1.push_back((int32_t)e);
    m.face_f1.push_back((int8_t)f);
    m.face_e2.push_back(-1 - bc);
    m.face_f2.push_back(0);
    m.nbr[f * K + e] = -1 - bc;
    m.nbrf[f * K + e] = 0;
    m.fid[f * K + e] = id;
  }
  m.F = (int64_t)m.face_e1.size();
  m.face_n.assign((size_t)dim * m.F, 0.0);
  m.face_sj.assign(m.F, 0.0);
  for (int64_t i = 0; i < m.F; ++i) {
    int64_t e = m.face_e1[i];
    int f = m.face_f1[i];
    for (int d = 0; d < dim; ++d) m.face_n[d * m.F + i] = m.fn[(f * dim + d) * K + e];
    m.face_sj[i] = m.fsj[f * K + e];
  }
  return true;
}

void build_bed_source(int dim, const RefOps& ops, int64_t K, const std::vector<double>& geo,
                      const std::vector<double>& bed, double gc, double gs, std::vector<double>& src) {
  const int NQ = ops.Nq, Np = ops.Np;
  src.assign((size_t)dim * NQ * K, 0.0);
  for (int64_t e = 0; e < K; ++e)
    for (int q = 0; q < NQ; ++q) {
      double Hr = 0.0, Hs = 0.0;
      for (int a = 0; a < Np; ++a) {
        Hr += ops.Drq[q * Np + a] * bed[e * Np + a];
        if (dim == 2) Hs += ops.Dsq[q * Np + a] * bed[e * Np + a];
      }
      double dHx = geo[e] * Hr;
      if (dim == 2) dHx += geo[2 * K + e] * Hs;
      src[(size_t)q * K + e] = -gc * dHx - gs;
      if (dim == 2) {
        const double dHy = geo[K + e] * Hr + geo[3 * K + e] * Hs;
        src[(size_t)(NQ + q) * K + e] = -gc * dHy;
      }
    }
}

}  // namespace dgswe
