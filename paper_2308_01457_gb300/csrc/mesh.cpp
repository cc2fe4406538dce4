// Host side of the library: error reporting, quadrature rules, RWG mesh tables
// (Section IV: lowest-order div-conforming elements on flat triangles) and the
// touching-pair list for the singular quadrature.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <set>

#include "fosb_internal.h"

namespace fosb {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};

void note_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }

fosb_status fail(fosb_status code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

fosb_status cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? FOSB_ERR_OOM : FOSB_ERR_CUDA;
}

// Symmetric 6-point degree-4 triangle rule (Dunavant 1985) from its closed form:
// nodes (a, a, 1-2a), (b, b, 1-2b), a, b = (8 - sqrt10 +- sqrt(38 - 44 sqrt(2/5)))/18,
// weights (620 +- sqrt(213125 - 53320 sqrt10))/3720.  Gauss-Legendre nodes on [0,1]
// by Newton's method on the three-term Legendre recurrence.
Rules make_rules(int nss) {
  Rules r{};
  const double s10 = std::sqrt(10.0);
  const double rt = std::sqrt(38.0 - 44.0 * std::sqrt(0.4));
  const double a = (8.0 - s10 + rt) / 18.0, b = (8.0 - s10 - rt) / 18.0;
  const double q = std::sqrt(213125.0 - 53320.0 * s10);
  const double wa = (620.0 + q) / 3720.0, wb = (620.0 - q) / 3720.0;
  const double pts[2] = {a, b}, wts[2] = {wa, wb};
  for (int g = 0; g < 2; ++g)
    for (int j = 0; j < 3; ++j) {
      int idx = 3 * g + j;
      for (int c = 0; c < 3; ++c) r.bary[idx][c] = (c == j) ? 1.0 - 2.0 * pts[g] : pts[g];
      r.w[idx] = wts[g];
    }
  r.nss = nss;
  for (int i = 0; i < nss; ++i) {
    double x = std::cos(M_PI * (i + 0.75) / (nss + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int n = 2; n <= nss; ++n) {
        double p2 = ((2.0 * n - 1.0) * x * p1 - (n - 1.0) * p0) / n;
        p0 = p1;
        p1 = p2;
      }
      double pn = nss == 1 ? x : p1;
      double pnm1 = nss == 1 ? 1.0 : p0;
      dp = nss * (x * pn - pnm1) / (x * x - 1.0);
      double dx = pn / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    // recompute derivative at the converged node
    double p0 = 1.0, p1 = x;
    for (int n = 2; n <= nss; ++n) {
      double p2 = ((2.0 * n - 1.0) * x * p1 - (n - 1.0) * p0) / n;
      p0 = p1;
      p1 = p2;
    }
    double pn = nss == 1 ? x : p1, pnm1 = nss == 1 ? 1.0 : p0;
    dp = nss * (x * pn - pnm1) / (x * x - 1.0);
    r.glx[i] = 0.5 * (1.0 - x);
    r.glw[i] = 1.0 / ((1.0 - x * x) * dp * dp);  // (2/((1-x^2) P'^2)) / 2
  }
  return r;
}

}  // namespace fosb

using namespace fosb;

namespace {

template <typename T>
fosb_status upload(T** dst, const void* src, size_t count) {
  if (count == 0) {
    *dst = nullptr;
    return FOSB_OK;
  }
  FOSB_CUDA(cudaMalloc(reinterpret_cast<void**>(dst), count * sizeof(T)));
  FOSB_CUDA(cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice));
  return FOSB_OK;
}

void free_dev(DevMesh& d) {
  void* ptrs[] = {d.verts,    d.vnormals,   d.tris,   d.tri_edge, d.tri_coef, d.tri_div,
                  d.tri_area, d.tri_normal, d.tri_qp, d.touch,    d.ell_cols, d.tri_ff};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  d = DevMesh{};
}

}  // namespace

extern "C" {

const char* fosb_last_error(void) { return g_last_error.c_str(); }

const char* fosb_version(void) { return "fosb-gb300 0.1 (sm_103a)"; }

uint64_t fosb_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

fosb_status fosb_mesh_create(const double* verts, int64_t nv, const int32_t* tris, int64_t nt, const double* vnormals,
                             fosb_mesh* out) {
  if (!verts || !tris || !out || nv < 3 || nt < 2) return fail(FOSB_ERR_INVALID_ARG, "fosb_mesh_create: bad arguments");
  if (nt > (int64_t(1) << 29)) return fail(FOSB_ERR_INVALID_ARG, "fosb_mesh_create: too many triangles");
  *out = nullptr;
  for (int64_t i = 0; i < 3 * nv; ++i)
    if (!std::isfinite(verts[i])) return fail(FOSB_ERR_MESH, "fosb_mesh_create: non-finite vertex coordinate");
  fosb_mesh m = new (std::nothrow) fosb_mesh_s;
  if (!m) return fail(FOSB_ERR_OOM, "fosb_mesh_create: host allocation");
  cudaGetDevice(&m->device);
  m->verts.assign(verts, verts + 3 * nv);
  m->tris.assign(tris, tris + 3 * nt);
  for (int64_t i = 0; i < 3 * nt; ++i)
    if (tris[i] < 0 || tris[i] >= nv) {
      delete m;
      return fail(FOSB_ERR_MESH, "fosb_mesh_create: vertex index out of range");
    }
  auto V = [&](int32_t i, int c) { return verts[3 * i + c]; };
  std::vector<double> area(nt), nrm(3 * nt);
  double max_edge = 0.0;
  for (int64_t t = 0; t < nt; ++t) {
    const int32_t* T = tris + 3 * t;
    double e1[3], e2[3];
    for (int c = 0; c < 3; ++c) {
      e1[c] = V(T[1], c) - V(T[0], c);
      e2[c] = V(T[2], c) - V(T[0], c);
    }
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    double l1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    double l2 = std::sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
    max_edge = std::max(max_edge, std::max(l1, l2));
    if (!(len > 1e-12 * l1 * l2) || T[0] == T[1] || T[1] == T[2] || T[0] == T[2]) {
      delete m;
      return fail(FOSB_ERR_MESH, "fosb_mesh_create: degenerate triangle " + std::to_string(t));
    }
    area[t] = 0.5 * len;
    for (int c = 0; c < 3; ++c) nrm[3 * t + c] = n[c] / len;
  }
  // edges: unordered pairs (a < b) in lexicographic order
  std::map<std::pair<int32_t, int32_t>, std::vector<std::pair<int64_t, int>>> emap;
  for (int64_t t = 0; t < nt; ++t)
    for (int i = 0; i < 3; ++i) {
      int32_t u = tris[3 * t + (i + 1) % 3], v = tris[3 * t + (i + 2) % 3];
      emap[{std::min(u, v), std::max(u, v)}].push_back({t, i});
    }
  const int64_t ne = int64_t(emap.size());
  m->edges.resize(2 * ne);
  m->edge_tris.resize(2 * ne);
  m->tri_edge.assign(3 * nt, -1);
  m->tri_sign.assign(3 * nt, 0.0);
  int64_t eidx = 0;
  for (auto& kv : emap) {
    auto& occ = kv.second;
    bool ok = occ.size() == 2;
    int plus = -1, minus = -1;
    if (ok) {
      for (int o = 0; o < 2; ++o) {
        int64_t t = occ[o].first;
        int i = occ[o].second;
        bool forward = tris[3 * t + (i + 1) % 3] == kv.first.first;  // runs a -> b
        (forward ? plus : minus) = o;
      }
      ok = plus >= 0 && minus >= 0;
    }
    if (!ok) {
      delete m;
      return fail(FOSB_ERR_MESH, "fosb_mesh_create: edge (" + std::to_string(kv.first.first) + "," +
                                     std::to_string(kv.first.second) +
                                     ") is not shared by exactly two oppositely oriented triangles");
    }
    m->edges[2 * eidx] = kv.first.first;
    m->edges[2 * eidx + 1] = kv.first.second;
    m->edge_tris[2 * eidx] = int32_t(occ[plus].first);
    m->edge_tris[2 * eidx + 1] = int32_t(occ[minus].first);
    m->tri_edge[3 * occ[plus].first + occ[plus].second] = int32_t(eidx);
    m->tri_sign[3 * occ[plus].first + occ[plus].second] = 1.0;
    m->tri_edge[3 * occ[minus].first + occ[minus].second] = int32_t(eidx);
    m->tri_sign[3 * occ[minus].first + occ[minus].second] = -1.0;
    ++eidx;
  }
  // vertex normals
  if (vnormals) {
    m->vnormals.assign(vnormals, vnormals + 3 * nv);
  } else {
    m->vnormals.assign(3 * nv, 0.0);
    for (int64_t t = 0; t < nt; ++t)
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) m->vnormals[3 * tris[3 * t + a] + c] += area[t] * nrm[3 * t + c];
    for (int64_t p = 0; p < nv; ++p) {
      double* n = &m->vnormals[3 * p];
      double l = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      if (l > 0)
        for (int c = 0; c < 3; ++c) n[c] /= l;
    }
  }
  // touching pairs t1 <= t2 with Sauter-Schwab vertex orderings:
  //   identical: stored order for both;
  //   edge: the shared edge as it runs (a -> b) in t1's cyclic order, then the third vertex;
  //   vertex: the shared vertex then the next two of each triangle's cyclic order.
  std::vector<std::vector<int32_t>> vtri(nv);
  for (int64_t t = 0; t < nt; ++t)
    for (int a = 0; a < 3; ++a) vtri[tris[3 * t + a]].push_back(int32_t(t));
  for (int64_t t1 = 0; t1 < nt; ++t1) {
    std::set<int32_t> nb;
    for (int a = 0; a < 3; ++a)
      for (int32_t t2 : vtri[tris[3 * t1 + a]])
        if (t2 >= t1) nb.insert(t2);
    const int32_t* A = tris + 3 * t1;
    for (int32_t t2 : nb) {
      const int32_t* B = tris + 3 * t2;
      TouchPair tp{};
      tp.t1 = int32_t(t1);
      tp.t2 = t2;
      if (t2 == t1) {
        tp.kind = 3;
        for (int s = 0; s < 3; ++s) tp.p[s] = tp.q[s] = A[s];
      } else {
        int inB[3], ns = 0;
        for (int i = 0; i < 3; ++i) {
          inB[i] = -1;
          for (int j = 0; j < 3; ++j)
            if (A[i] == B[j]) inB[i] = j;
          ns += inB[i] >= 0;
        }
        if (ns == 1) {
          int i = inB[0] >= 0 ? 0 : (inB[1] >= 0 ? 1 : 2), j = inB[i];
          tp.kind = 1;
          for (int s = 0; s < 3; ++s) {
            tp.p[s] = A[(i + s) % 3];
            tp.q[s] = B[(j + s) % 3];
          }
        } else if (ns == 2) {
          int i0 = 0;
          for (int i = 0; i < 3; ++i)
            if (inB[i] >= 0 && inB[(i + 1) % 3] >= 0) i0 = i;
          int32_t a = A[i0], b = A[(i0 + 1) % 3], c1 = A[(i0 + 2) % 3], c2 = -1;
          for (int j = 0; j < 3; ++j)
            if (B[j] != a && B[j] != b) c2 = B[j];
          tp.kind = 2;
          tp.p[0] = a; tp.p[1] = b; tp.p[2] = c1;
          tp.q[0] = a; tp.q[1] = b; tp.q[2] = c2;
        } else {
          delete m;
          return fail(FOSB_ERR_MESH, "fosb_mesh_create: duplicated triangle");
        }
      }
      m->touch.push_back(tp);
    }
  }
  // per-triangle records
  Rules r = make_rules(5);
  std::vector<double> coef(3 * nt), dv(3 * nt), qp(18 * nt);
  std::vector<double> len(ne);
  for (int64_t e = 0; e < ne; ++e) {
    double s = 0;
    for (int c = 0; c < 3; ++c) {
      double d = V(m->edges[2 * e + 1], c) - V(m->edges[2 * e], c);
      s += d * d;
    }
    len[e] = std::sqrt(s);
  }
  for (int64_t t = 0; t < nt; ++t) {
    for (int i = 0; i < 3; ++i) {
      double l = len[m->tri_edge[3 * t + i]], s = m->tri_sign[3 * t + i];
      coef[3 * t + i] = s * l / (2.0 * area[t]);
      dv[3 * t + i] = s * l / area[t];
    }
    for (int q = 0; q < 6; ++q)
      for (int c = 0; c < 3; ++c)
        qp[18 * t + 3 * q + c] = r.bary[q][0] * V(tris[3 * t], c) + r.bary[q][1] * V(tris[3 * t + 1], c) +
                                 r.bary[q][2] * V(tris[3 * t + 2], c);
  }
  // ELL columns of the shape-derivative matrix: the four vertices in the support of f_m
  std::vector<int32_t> ell(4 * ne);
  for (int64_t e = 0; e < ne; ++e) {
    ell[4 * e] = m->edges[2 * e];
    ell[4 * e + 1] = m->edges[2 * e + 1];
    for (int s = 0; s < 2; ++s) {
      int32_t t = m->edge_tris[2 * e + s];
      for (int a = 0; a < 3; ++a)
        if (m->tri_edge[3 * t + a] == e) ell[4 * e + 2 + s] = tris[3 * t + a];
    }
  }
  // float-float per-triangle fields (hi = nearest float, lo = nearest float of the rest)
  std::vector<float> tff(size_t(kTriFF) * nt);
  auto put = [&](int f, int64_t t, double x) {
    float h = float(x);
    tff[size_t(f) * nt + t] = h;
    tff[size_t(f + 1) * nt + t] = float(x - double(h));
  };
  double lo3[3] = {1e300, 1e300, 1e300}, hi3[3] = {-1e300, -1e300, -1e300};
  for (int64_t p = 0; p < nv; ++p)
    for (int c = 0; c < 3; ++c) {
      lo3[c] = std::min(lo3[c], verts[3 * p + c]);
      hi3[c] = std::max(hi3[c], verts[3 * p + c]);
    }
  for (int64_t t = 0; t < nt; ++t) {
    const int32_t* T = tris + 3 * t;
    for (int q = 0; q < 6; ++q)
      for (int c = 0; c < 3; ++c) put((q * 3 + c) * 2, t, qp[18 * t + 3 * q + c] - V(T[0], c));
    for (int c = 0; c < 3; ++c) {
      put(36 + 2 * c, t, V(T[0], c));
      put(42 + 2 * c, t, V(T[1], c) - V(T[0], c));
      put(48 + 2 * c, t, V(T[2], c) - V(T[0], c));
    }
    for (int i = 0; i < 3; ++i) put(54 + 2 * i, t, m->tri_sign[3 * t + i] * len[m->tri_edge[3 * t + i]]);
  }
  DevMesh& d = m->d;
  d.diameter = std::sqrt((hi3[0] - lo3[0]) * (hi3[0] - lo3[0]) + (hi3[1] - lo3[1]) * (hi3[1] - lo3[1]) +
                         (hi3[2] - lo3[2]) * (hi3[2] - lo3[2]));
  d.nv = nv;
  d.nt = nt;
  d.ne = ne;
  d.ntouch = int64_t(m->touch.size());
  fosb_status st = FOSB_OK;
  if ((st = upload(&d.verts, verts, 3 * nv)) || (st = upload(&d.vnormals, m->vnormals.data(), 3 * nv)) ||
      (st = upload(&d.tris, tris, 3 * nt)) || (st = upload(&d.tri_edge, m->tri_edge.data(), 3 * nt)) ||
      (st = upload(&d.tri_coef, coef.data(), 3 * nt)) || (st = upload(&d.tri_div, dv.data(), 3 * nt)) ||
      (st = upload(&d.tri_area, area.data(), nt)) || (st = upload(&d.tri_normal, nrm.data(), 3 * nt)) ||
      (st = upload(&d.tri_qp, qp.data(), 18 * nt)) || (st = upload(&d.touch, m->touch.data(), m->touch.size())) ||
      (st = upload(&d.ell_cols, ell.data(), 4 * ne)) || (st = upload(&d.tri_ff, tff.data(), tff.size()))) {
    free_dev(d);
    delete m;
    return st;
  }
  *out = m;
  return FOSB_OK;
}

fosb_status fosb_mesh_info(fosb_mesh m, int64_t* nv, int64_t* nt, int64_t* n_edges, int64_t* n_touching) {
  if (!m) return fail(FOSB_ERR_INVALID_ARG, "fosb_mesh_info: NULL mesh");
  if (nv) *nv = m->d.nv;
  if (nt) *nt = m->d.nt;
  if (n_edges) *n_edges = m->d.ne;
  if (n_touching) *n_touching = m->d.ntouch;
  return FOSB_OK;
}

fosb_status fosb_mesh_edges(fosb_mesh m, int32_t* edges, int32_t* edge_tris) {
  if (!m) return fail(FOSB_ERR_INVALID_ARG, "fosb_mesh_edges: NULL mesh");
  if (edges) std::memcpy(edges, m->edges.data(), m->edges.size() * sizeof(int32_t));
  if (edge_tris) std::memcpy(edge_tris, m->edge_tris.data(), m->edge_tris.size() * sizeof(int32_t));
  return FOSB_OK;
}

fosb_status fosb_mesh_destroy(fosb_mesh m) {
  if (!m) return FOSB_OK;
  free_dev(m->d);
  delete m;
  return FOSB_OK;
}

}  // extern "C"
