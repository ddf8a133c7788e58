// TEST INFRASTRUCTURE — the oracle. Not part of the product path.
//
// A plain, slow, sequential CPU restatement of SLIM-VDB scan integration
// (arXiv 2512.12945), written from the paper's definitions:
//   * Sec. III-A "Surface Reconstruction": truncated-band raycasting and the
//     weighted running average of the truncated signed distance (equation for
//     D_t and Eq. (Wx) for W_t, with the weighting function w~ = 1).
//   * Sec. III-C "Closed-Set Semantic Fusion": Theorem 1 / Eq. (alpha_update)
//     Dirichlet count update, Eq. (dir_to_cat) posterior predictive; and the
//     non-Bayesian ablation of Sec. IV (SLIM-VDB*): the latest label wins.
//   * Sec. III-D "Open-Set Semantic Fusion": Theorem 2 / Eqs. (norm_update_1)
//     to (norm_update_4) Normal-Inverse-Gamma update, with the implementation
//     simplification stated at the end of Sec. III-D (lambda = 2 nu = W, only
//     the diagonal beta is tracked), and the cosine-similarity / softmax /
//     T_p = 0.1 threshold read-out.
//
// Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline may load
// this library. It shares no code with the CUDA path.
//
// Geometry (transform, DDA, per-pair SDF) follows a fixed FP32 operation
// order so that voxel key sets are reproducible bit for bit: every operation
// is one IEEE-754 round-to-nearest float op, no fused multiply-add (the file
// is compiled with -ffp-contract=off and without fast-math). All fusion
// arithmetic (TSDF, Dirichlet counts, NIG) is done in FP64, one observation
// (voxel, point pair) at a time, in scan order, then point order, then ray
// order. A second mode (fp64_geometry = 1) runs the geometry in FP64 too; it
// is used only to state the error of the FP32 geometry.
//
// Readings where the paper is silent (the DDA is Amanatides & Woo 1987, the
// SDF is the projective along-ray distance, the band is [r - tau, r + tau]
// clipped at the sensor, tau and the voxel size are in metres, every voxel of
// the band receives the semantic observation, priors alpha0 >= 0 and
// m0 = lambda0 = nu0 = beta0 = 0) are listed in the design notes of the repo.

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <unordered_map>
#include <vector>

namespace {

enum Mode : int32_t { CLOSED_ONEHOT = 0, CLOSED_SOFT = 1, OPEN = 2, CLOSED_LATEST = 3 };

struct Params {
  float voxel_size;
  float trunc;
  float min_range;
  float max_range;
  int32_t mode;
  int32_t num_classes;
  int32_t embed_dim;
  int32_t fp64_geometry;
  double alpha0;
  double body_from_sensor[16];  // row-major 4x4
  int32_t weighting;  // 0: w~ = 1; 1: linear decay behind the surface
  float weight_eps;   // linear decay: w~ = 1 for d >= -eps (0 <= eps < tau)
};

struct VKey {
  int32_t x, y, z;
  bool operator==(const VKey& o) const { return x == o.x && y == o.y && z == o.z; }
};

struct VKeyHash {
  size_t operator()(const VKey& k) const {
    uint64_t h = (uint64_t)(uint32_t)k.x * 0x9E3779B97F4A7C15ull;
    h ^= (uint64_t)(uint32_t)k.y * 0xC2B2AE3D27D4EB4Full + (h << 6) + (h >> 2);
    h ^= (uint64_t)(uint32_t)k.z * 0x165667B19E3779F9ull + (h << 6) + (h >> 2);
    return (size_t)h;
  }
};

// One voxel's state. D and W: Sec. III-A. sem: Dirichlet counts c_i
// (alpha_i - alpha0) in closed-set modes, the NIG mean m in open-set mode.
// beta: the NIG beta (open set only).
struct Rec {
  double D = 0.0;
  double W = 0.0;
  std::vector<double> sem;
  std::vector<double> beta;
};

struct Map {
  Params p;
  std::unordered_map<VKey, Rec, VKeyHash> vox;
  std::vector<VKey> order;  // extract order, filled by ora_extract
};

// One (voxel, point) observation of a scan.
struct Pair {
  int32_t i[3];
  double d;
};

// Floor division by 8 (block coordinate of a voxel index), written plainly.
int32_t block_of(int32_t i) { return (int32_t)std::floor((double)i / 8.0); }

int32_t local_of(const int32_t i[3]) {
  int32_t lx = i[0] - 8 * block_of(i[0]);
  int32_t ly = i[1] - 8 * block_of(i[1]);
  int32_t lz = i[2] - 8 * block_of(i[2]);
  return (lx * 8 + ly) * 8 + lz;
}

// world_from_sensor = world_from_body * body_from_sensor, in FP64.
void compose(const double pose[16], const double ext[16], double out[16]) {
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += pose[r * 4 + k] * ext[k * 4 + c];
      out[r * 4 + c] = s;
    }
}

// Cap on the number of voxels one ray band may visit: 3 * ceil(2 tau / v) + 3.
int step_cap(float v, float tau) {
  return 3 * (int)std::ceil(2.0 * (double)tau / (double)v) + 3;
}

// ---------------------------------------------------------------- FP32 path
// Point validity, transform and the band DDA for one point, each float
// operation written as its own statement (round to nearest, no FMA).
// visits: every voxel the DDA enters (before the SDF filter).
// pairs:  the observations kept after the SDF filter (d >= -tau, d <= tau).
// Returns false when the point is invalid.
bool point_pairs_f32(const Params& P, const float R[9], const float t[3],
                     const float p[3], std::vector<std::array<int32_t, 3>>* visits,
                     std::vector<Pair>* pairs) {
  const float v = P.voxel_size, tau = P.trunc;
  if (!std::isfinite(p[0]) || !std::isfinite(p[1]) || !std::isfinite(p[2])) return false;
  // sensor-frame range
  float q0 = p[0] * p[0];
  float q1 = p[1] * p[1];
  float q2 = p[2] * p[2];
  float qs = q0 + q1;
  qs = qs + q2;
  float rs = std::sqrt(qs);
  if (!(rs >= P.min_range && rs <= P.max_range)) return false;
  // x = R p + t
  float x[3];
  for (int a = 0; a < 3; ++a) {
    float m0 = R[a * 3 + 0] * p[0];
    float m1 = R[a * 3 + 1] * p[1];
    float m2 = R[a * 3 + 2] * p[2];
    float s = m0 + m1;
    s = s + m2;
    x[a] = s + t[a];
  }
  const float lim = 524288.0f * v;  // 2^19 voxels from the world origin
  for (int a = 0; a < 3; ++a) {
    if (!(std::fabs(x[a]) < lim)) return false;
    if (!(std::fabs(t[a]) < lim)) return false;
  }
  // ray from the sensor origin o = t
  float dl[3], u[3];
  for (int a = 0; a < 3; ++a) dl[a] = x[a] - t[a];
  float r0 = dl[0] * dl[0];
  float r1 = dl[1] * dl[1];
  float r2 = dl[2] * dl[2];
  float rr = r0 + r1;
  rr = rr + r2;
  float r = std::sqrt(rr);
  if (!(r > 0.0f) || !std::isfinite(r)) return false;
  for (int a = 0; a < 3; ++a) u[a] = dl[a] / r;

  // Amanatides & Woo traversal of t in [t0, t1].
  float t0 = r - tau;
  if (t0 < 0.0f) t0 = 0.0f;
  float t1 = r + tau;
  int32_t ii[3], step[3];
  float tMax[3], tDelta[3];
  for (int a = 0; a < 3; ++a) {
    float tu = t0 * u[a];
    float s = t[a] + tu;
    float sv = s / v;
    ii[a] = (int32_t)std::floor(sv);
    step[a] = u[a] > 0.0f ? 1 : (u[a] < 0.0f ? -1 : 0);
    if (u[a] != 0.0f) {
      tDelta[a] = v / std::fabs(u[a]);
      float bnd = (float)(ii[a] + (step[a] > 0 ? 1 : 0)) * v;
      float gap = bnd - s;
      float dt = gap / u[a];
      tMax[a] = t0 + dt;
    } else {
      tDelta[a] = INFINITY;
      tMax[a] = INFINITY;
    }
  }
  const int cap = step_cap(v, tau);
  for (int k = 0; k < cap; ++k) {
    if (visits) visits->push_back({ii[0], ii[1], ii[2]});
    // signed distance of the voxel centre along the ray
    float c[3], e[3];
    for (int a = 0; a < 3; ++a) {
      float fi = (float)ii[a] + 0.5f;
      c[a] = fi * v;
      e[a] = x[a] - c[a];
    }
    float d0 = e[0] * u[0];
    float d1 = e[1] * u[1];
    float d2 = e[2] * u[2];
    float d = d0 + d1;
    d = d + d2;
    if (pairs && !(d < -tau)) {
      if (d > tau) d = tau;
      Pair pr;
      pr.i[0] = ii[0];
      pr.i[1] = ii[1];
      pr.i[2] = ii[2];
      pr.d = (double)d;
      pairs->push_back(pr);
    }
    int a = 0;
    if (tMax[1] < tMax[a]) a = 1;
    if (tMax[2] < tMax[a]) a = 2;
    if (tMax[a] > t1) break;
    ii[a] += step[a];
    tMax[a] = tMax[a] + tDelta[a];
  }
  return true;
}

// ---------------------------------------------------------------- FP64 path
// Same steps in double precision (used only to state the FP32 error).
bool point_pairs_f64(const Params& P, const double M[16], const float pf[3],
                     std::vector<std::array<int32_t, 3>>* visits,
                     std::vector<Pair>* pairs) {
  const double v = P.voxel_size, tau = P.trunc;
  double p[3] = {pf[0], pf[1], pf[2]};
  if (!std::isfinite(p[0]) || !std::isfinite(p[1]) || !std::isfinite(p[2])) return false;
  double rs = std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  if (!(rs >= P.min_range && rs <= P.max_range)) return false;
  double x[3], o[3];
  for (int a = 0; a < 3; ++a) {
    x[a] = M[a * 4 + 0] * p[0] + M[a * 4 + 1] * p[1] + M[a * 4 + 2] * p[2] + M[a * 4 + 3];
    o[a] = M[a * 4 + 3];
  }
  const double lim = 524288.0 * v;
  for (int a = 0; a < 3; ++a)
    if (!(std::fabs(x[a]) < lim) || !(std::fabs(o[a]) < lim)) return false;
  double dl[3] = {x[0] - o[0], x[1] - o[1], x[2] - o[2]};
  double r = std::sqrt(dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2]);
  if (!(r > 0.0)) return false;
  double u[3] = {dl[0] / r, dl[1] / r, dl[2] / r};
  double t0 = std::max(0.0, r - tau), t1 = r + tau;
  int32_t ii[3], step[3];
  double tMax[3], tDelta[3];
  for (int a = 0; a < 3; ++a) {
    double s = o[a] + t0 * u[a];
    ii[a] = (int32_t)std::floor(s / v);
    step[a] = u[a] > 0 ? 1 : (u[a] < 0 ? -1 : 0);
    if (u[a] != 0) {
      tDelta[a] = v / std::fabs(u[a]);
      tMax[a] = t0 + ((ii[a] + (step[a] > 0 ? 1 : 0)) * v - s) / u[a];
    } else {
      tDelta[a] = INFINITY;
      tMax[a] = INFINITY;
    }
  }
  const int cap = step_cap(P.voxel_size, P.trunc);
  for (int k = 0; k < cap; ++k) {
    if (visits) visits->push_back({ii[0], ii[1], ii[2]});
    double d = 0;
    for (int a = 0; a < 3; ++a) d += (x[a] - (ii[a] + 0.5) * v) * u[a];
    if (pairs && !(d < -tau)) {
      Pair pr;
      pr.i[0] = ii[0];
      pr.i[1] = ii[1];
      pr.i[2] = ii[2];
      pr.d = std::min(d, tau);
      pairs->push_back(pr);
    }
    int a = 0;
    if (tMax[1] < tMax[a]) a = 1;
    if (tMax[2] < tMax[a]) a = 2;
    if (tMax[a] > t1) break;
    ii[a] += step[a];
    tMax[a] += tDelta[a];
  }
  return true;
}

void pose_f32(const Params& P, const double pose[16], float R[9], float t[3], double M[16]) {
  compose(pose, P.body_from_sensor, M);
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) R[a * 3 + b] = (float)M[a * 4 + b];
    t[a] = (float)M[a * 4 + 3];
  }
}

bool point_pairs(const Params& P, const float R[9], const float t[3], const double M[16],
                 const float p[3], std::vector<std::array<int32_t, 3>>* visits,
                 std::vector<Pair>* pairs) {
  if (P.fp64_geometry) return point_pairs_f64(P, M, p, visits, pairs);
  return point_pairs_f32(P, R, t, p, visits, pairs);
}

int sem_width(const Params& P) { return P.mode == OPEN ? P.embed_dim : P.num_classes; }

// Index of the largest probability; ties go to the lowest index.
int argmax_first(const float* p, int K) {
  int best = 0;
  for (int k = 1; k < K; ++k)
    if (p[k] > p[best]) best = k;
  return best;
}

// The weight w~ of an observation with SDF d (Sec. III-A leaves the weighting
// function open and names w~ = 1 as the common choice). weighting = 1 is the
// linear decay behind the surface of Bylow et al. (RSS 2013), in this
// code's sign convention (d > 0 in front of the surface): w~ = 1 for
// d >= -eps, falling linearly to 0 at d = -tau.
double obs_weight(const Params& P, double d) {
  if (P.weighting == 0 || d >= -(double)P.weight_eps) return 1.0;
  return ((double)P.trunc + d) / ((double)P.trunc - (double)P.weight_eps);
}

// Fuse one observation (d, semantic measurement) into a voxel.
void fuse(const Params& P, Rec& rec, double d, const float* s) {
  const double W_prev = rec.W;
  // Sec. III-A: W_t = W_{t-1} + w~, D_t = (W_{t-1} D_{t-1} + w~ d) / W_t.
  const double wt = obs_weight(P, d);
  rec.W = W_prev + wt;
  rec.D = (W_prev * rec.D + wt * d) / rec.W;
  if (P.mode == CLOSED_ONEHOT) {
    // Theorem 1, Eq. (alpha_update): alpha_i += 1{z = i}, z = argmax of the
    // network's class probabilities (one-hot prediction); a weighted
    // observation adds w~ (w~ = 1 is the paper's update).
    rec.sem[argmax_first(s, P.num_classes)] += wt;
  } else if (P.mode == CLOSED_SOFT) {
    // Soft-count reading of Eq. (alpha_update): alpha_i += w~ p_i.
    for (int k = 0; k < P.num_classes; ++k) rec.sem[k] += wt * (double)s[k];
  } else if (P.mode == CLOSED_LATEST) {
    // The non-Bayesian ablation of the evaluation (SLIM-VDB*): the voxel
    // keeps the most recent measurement's label, as a one-hot vector.
    std::fill(rec.sem.begin(), rec.sem.end(), 0.0);
    rec.sem[argmax_first(s, P.num_classes)] = 1.0;
  } else {
    // Theorem 2 with |Z| = 1 and lambda = W_prev (Sec. III-D):
    //   m~ = (lambda m + z) / (lambda + 1)
    //   beta~ = beta + (lambda / (lambda + 1)) (z - m)^2 / 2
    const double lam = W_prev, lam_new = W_prev + 1.0;
    for (int k = 0; k < P.embed_dim; ++k) {
      const double z = (double)s[k];
      const double m_old = rec.sem[k];
      rec.sem[k] = (lam * m_old + z) / lam_new;
      rec.beta[k] += (lam / lam_new) * (z - m_old) * (z - m_old) * 0.5;
    }
  }
}

bool key_less(const VKey& a, const VKey& b) {
  int32_t ia[3] = {a.x, a.y, a.z}, ib[3] = {b.x, b.y, b.z};
  for (int k = 0; k < 3; ++k) {
    int32_t ba = block_of(ia[k]), bb = block_of(ib[k]);
    if (ba != bb) return ba < bb;
  }
  return local_of(ia) < local_of(ib);
}

}  // namespace

extern "C" {

typedef Params ora_params;

// Returns null for an unsupported combination: a weighting other than
// w~ = 1 applies to the closed-set modes only (the open-set update ties the
// NIG lambda to W, Sec. III-D).
void* ora_create(const ora_params* p) {
  if (p->weighting != 0 && (p->mode == OPEN || p->weighting != 1 ||
                            !(p->weight_eps >= 0.0f && p->weight_eps < p->trunc)))
    return nullptr;
  Map* m = new Map();
  m->p = *p;
  return m;
}

void ora_destroy(void* h) { delete (Map*)h; }

// Integrate one scan: n sensor-frame points (n x 3 float), the body pose
// (row-major 4x4 double, world_from_body) and per-point semantics (n x K
// class probabilities, or n x l embeddings). Returns the number of valid
// points.
int64_t ora_integrate(void* h, const float* pts, int64_t n, const double pose[16],
                      const float* sem) {
  Map& m = *(Map*)h;
  const Params& P = m.p;
  float R[9], t[3];
  double M[16];
  pose_f32(P, pose, R, t, M);
  const int w = sem_width(P);
  std::vector<Pair> pairs;
  int64_t valid = 0;
  for (int64_t j = 0; j < n; ++j) {
    pairs.clear();
    if (!point_pairs(P, R, t, M, pts + 3 * j, nullptr, &pairs)) continue;
    ++valid;
    const float* s = sem + (size_t)j * (size_t)w;
    for (const Pair& pr : pairs) {
      // an observation of weight 0 (d = -tau under the linear decay) changes
      // nothing: a voxel is in the map once its weight W is positive
      if (obs_weight(P, pr.d) == 0.0) continue;
      VKey key{pr.i[0], pr.i[1], pr.i[2]};
      auto it = m.vox.find(key);
      if (it == m.vox.end()) {
        Rec rec;
        rec.sem.assign((size_t)w, 0.0);
        if (P.mode == OPEN) rec.beta.assign((size_t)w, 0.0);
        it = m.vox.emplace(key, std::move(rec)).first;
      }
      fuse(P, it->second, pr.d, s);
    }
  }
  return valid;
}

// Integrate one depth frame (the RGB-D front end): pixel (u, v) of a
// row-major width x height z-depth image (metres along the camera's optical
// axis) back-projects, in FP32 with this op order, to the sensor-frame point
// p = (((u + 0.5) - cx) / fx * z, ((v + 0.5) - cy) / fy * z, z); pixels with
// a non-finite or non-positive z are invalid. The points then go through
// ora_integrate unchanged (sem: one row per pixel). Returns the number of
// valid points.
int64_t ora_integrate_depth(void* h, const float* depth, int32_t width, int32_t height, float fx,
                            float fy, float cx, float cy, const double pose[16],
                            const float* sem) {
  const int64_t n = (int64_t)width * height;
  std::vector<float> pts((size_t)n * 3);
  for (int32_t v = 0; v < height; ++v)
    for (int32_t u = 0; u < width; ++u) {
      const int64_t j = (int64_t)v * width + u;
      const float z = depth[j];
      if (!(z > 0.0f) || !std::isfinite(z)) {
        pts[3 * j + 0] = pts[3 * j + 1] = pts[3 * j + 2] = NAN;
        continue;
      }
      float au = (float)u + 0.5f;
      float av = (float)v + 0.5f;
      float xu = (au - cx) / fx;
      float yv = (av - cy) / fy;
      pts[3 * j + 0] = xu * z;
      pts[3 * j + 1] = yv * z;
      pts[3 * j + 2] = z;
    }
  return ora_integrate(h, pts.data(), n, pose, sem);
}

// All (voxel, point) observations of one scan, in point then ray order.
// Returns the number of pairs (or the required count when cap is too small).
int64_t ora_scan_pairs(const ora_params* p, const float* pts, int64_t n, const double pose[16],
                       int32_t* ijk, int64_t* pt, double* d, int64_t cap) {
  float R[9], t[3];
  double M[16];
  pose_f32(*p, pose, R, t, M);
  std::vector<Pair> pairs;
  int64_t k = 0;
  for (int64_t j = 0; j < n; ++j) {
    pairs.clear();
    if (!point_pairs(*p, R, t, M, pts + 3 * j, nullptr, &pairs)) continue;
    for (const Pair& pr : pairs) {
      if (k < cap) {
        for (int a = 0; a < 3; ++a) ijk[3 * k + a] = pr.i[a];
        pt[k] = j;
        d[k] = pr.d;
      }
      ++k;
    }
  }
  return k;
}

// Every voxel the band DDA of one point enters (before the SDF filter).
// Returns the count, or -1 for an invalid point.
int64_t ora_point_visits(const ora_params* p, const float pt[3], const double pose[16],
                         int32_t* ijk, int64_t cap) {
  float R[9], t[3];
  double M[16];
  pose_f32(*p, pose, R, t, M);
  std::vector<std::array<int32_t, 3>> vis;
  if (!point_pairs(*p, R, t, M, pt, &vis, nullptr)) return -1;
  int64_t k = 0;
  for (auto& a : vis) {
    if (k < cap)
      for (int c = 0; c < 3; ++c) ijk[3 * k + c] = a[c];
    ++k;
  }
  return k;
}

int64_t ora_count(void* h) { return (int64_t)((Map*)h)->vox.size(); }

// Allocated voxels sorted by (block x, block y, block z, local index) with
// local = ((i_x mod 8) * 8 + (i_y mod 8)) * 8 + (i_z mod 8).
// sem: n x K counts (or posteriors when posterior != 0), or n x l means.
// beta: n x l (open set; may be null).
int64_t ora_extract(void* h, int32_t* ijk, double* D, double* W, double* sem, double* beta,
                    int32_t posterior) {
  Map& m = *(Map*)h;
  const Params& P = m.p;
  m.order.clear();
  for (auto& kv : m.vox) m.order.push_back(kv.first);
  std::sort(m.order.begin(), m.order.end(), key_less);
  const int w = sem_width(P);
  for (size_t j = 0; j < m.order.size(); ++j) {
    const VKey& k = m.order[j];
    const Rec& r = m.vox.at(k);
    if (ijk) {
      ijk[3 * j + 0] = k.x;
      ijk[3 * j + 1] = k.y;
      ijk[3 * j + 2] = k.z;
    }
    if (D) D[j] = r.D;
    if (W) W[j] = r.W;
    if (sem) {
      if (P.mode != OPEN && P.mode != CLOSED_LATEST && posterior) {
        // Eq. (dir_to_cat): p(z = i) = alpha~_i / sum_j alpha~_j, with
        // alpha~_i = alpha0 + c_i.
        double tot = 0.0;
        for (int c = 0; c < w; ++c) tot += P.alpha0 + r.sem[c];
        for (int c = 0; c < w; ++c) sem[j * w + c] = (P.alpha0 + r.sem[c]) / tot;
      } else {
        for (int c = 0; c < w; ++c) sem[j * w + c] = r.sem[c];
      }
    }
    if (beta && P.mode == OPEN)
      for (int c = 0; c < w; ++c) beta[j * w + c] = r.beta[c];
  }
  return (int64_t)m.order.size();
}

// Uncertainty read-out, in the order of ora_extract (the map is re-sorted
// here). Closed set (Sec. III-C: the Dirichlet posterior Dir(alpha~) with
// alpha~_i = alpha0 + c_i, A = sum_i alpha~_i): unc is n x (K + 1), first
// the variance of each class probability, alpha~_i (A - alpha~_i) /
// (A^2 (A + 1)), then the entropy -sum_i p_i ln p_i of the posterior
// predictive p_i = alpha~_i / A (Eq. dir_to_cat; a zero p_i adds nothing).
// Open set (Eq. student_t): the predictive of each element is a Student-t
// with 2 nu degrees of freedom, location m and scale^2 beta (lambda + 1) /
// (lambda nu); its variance 2 nu / (2 nu - 2) * scale^2 exists for 2 nu > 2.
// With lambda = 2 nu = W (end of Sec. III-D) that is
// 2 beta (W + 1) / (W (W - 2)); unc is n x l, +inf where W <= 2.
int64_t ora_uncertainty(void* h, double* unc) {
  Map& m = *(Map*)h;
  const Params& P = m.p;
  std::vector<VKey> order;
  for (auto& kv : m.vox) order.push_back(kv.first);
  std::sort(order.begin(), order.end(), key_less);
  const int w = sem_width(P);
  for (size_t j = 0; j < order.size(); ++j) {
    const Rec& r = m.vox.at(order[j]);
    if (P.mode != OPEN) {
      double A = 0.0;
      for (int c = 0; c < w; ++c) A += P.alpha0 + r.sem[c];
      double H = 0.0;
      for (int c = 0; c < w; ++c) {
        const double a = P.alpha0 + r.sem[c];
        unc[j * (w + 1) + c] = a * (A - a) / (A * A * (A + 1.0));
        const double p = a / A;
        if (p > 0.0) H -= p * std::log(p);
      }
      unc[j * (w + 1) + w] = H;
    } else {
      const double lam = r.W, nu = r.W / 2.0;
      for (int c = 0; c < w; ++c) {
        if (!(2.0 * nu > 2.0)) {
          unc[j * w + c] = INFINITY;
          continue;
        }
        const double scale2 = r.beta[c] * (lam + 1.0) / (lam * nu);
        unc[j * w + c] = 2.0 * nu / (2.0 * nu - 2.0) * scale2;
      }
    }
  }
  return (int64_t)order.size();
}

// ----------------------------------------------------------------- render
// Voxels a ray o + t u enters for t in [t0, t1], in order (Amanatides & Woo,
// the same FP32 operation order as the band traversal of point_pairs_f32,
// ties to the lowest axis), at most cap of them.
void ray_visits_f32(float v, const float o[3], const float u[3], float t0, float t1, int cap,
                    std::vector<std::array<int32_t, 3>>* out) {
  int32_t ii[3], step[3];
  float tMax[3], tDelta[3];
  for (int a = 0; a < 3; ++a) {
    float tu = t0 * u[a];
    float s = o[a] + tu;
    float sv = s / v;
    ii[a] = (int32_t)std::floor(sv);
    step[a] = u[a] > 0.0f ? 1 : (u[a] < 0.0f ? -1 : 0);
    if (u[a] != 0.0f) {
      tDelta[a] = v / std::fabs(u[a]);
      float bnd = (float)(ii[a] + (step[a] > 0 ? 1 : 0)) * v;
      float gap = bnd - s;
      float dt = gap / u[a];
      tMax[a] = t0 + dt;
    } else {
      tDelta[a] = INFINITY;
      tMax[a] = INFINITY;
    }
  }
  for (int k = 0; k < cap; ++k) {
    out->push_back({ii[0], ii[1], ii[2]});
    int a = 0;
    if (tMax[1] < tMax[a]) a = 1;
    if (tMax[2] < tMax[a]) a = 2;
    if (tMax[a] > t1) break;
    ii[a] += step[a];
    tMax[a] = tMax[a] + tDelta[a];
  }
}

// Unit-length camera ray of pixel (px, py) of a pinhole camera (x right,
// y down, looking along +z), rotated into the world: FP32, fixed op order.
void pixel_ray_f32(const float R[9], float fx, float fy, float cx, float cy, int32_t px,
                   int32_t py, float u[3]) {
  float ax = (float)px + 0.5f;
  float ay = (float)py + 0.5f;
  float dx = (ax - cx) / fx;
  float dy = (ay - cy) / fy;
  float n2 = dx * dx;
  float m2 = dy * dy;
  n2 = n2 + m2;
  n2 = n2 + 1.0f;
  float nn = std::sqrt(n2);
  float d[3] = {dx / nn, dy / nn, 1.0f / nn};
  for (int a = 0; a < 3; ++a) {
    float m0 = R[a * 3 + 0] * d[0];
    float m1 = R[a * 3 + 1] * d[1];
    float m2a = R[a * 3 + 2] * d[2];
    float s = m0 + m1;
    u[a] = s + m2a;
  }
}

// Ray-cast render of the map from a pinhole camera (Sec. III-E: the map is
// rendered from a camera viewpoint instead of being meshed). Per pixel
// (row-major), the ray from the camera centre enters voxels for t in
// [near, far] (at most 3 ceil((far - near) / v) + 3 of them). A voxel is
// observed when the map holds it; its ray parameter is the projection of
// its centre, t_c = (c - o) . u (FP32). The surface is the first pair of
// consecutive entered voxels, both observed, with D_prev > 0 >= D: depth =
// t_prev + (t_c - t_prev) D_prev / (D_prev - D). Outputs at that voxel
// (the one with D <= 0): its indices, the closed-set label (the largest
// count, ties to the lowest class) or -1 for the open set, and for the open
// set with a query q the cosine m . q / (|m| |q|) (0 for a zero norm).
// A pixel without a crossing gets depth +inf, indices INT32_MIN, label -1,
// sim 0.
int64_t ora_render(void* h, const double world_from_camera[16], float fx, float fy, float cx,
                   float cy, int32_t width, int32_t height, float near_t, float far_t,
                   const float* q, double* depth, int32_t* ijk, int32_t* label, double* sim) {
  Map& m = *(Map*)h;
  const Params& P = m.p;
  const float v = P.voxel_size;
  float R[9], o[3];
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) R[a * 3 + b] = (float)world_from_camera[a * 4 + b];
    o[a] = (float)world_from_camera[a * 4 + 3];
  }
  const int cap = 3 * (int)std::ceil(((double)far_t - (double)near_t) / (double)v) + 3;
  const int w = sem_width(P);
  double qn = 0.0;
  if (q)
    for (int c = 0; c < w; ++c) qn += (double)q[c] * (double)q[c];
  qn = std::sqrt(qn);
  int64_t hits = 0;
  std::vector<std::array<int32_t, 3>> vis;
  for (int32_t py = 0; py < height; ++py)
    for (int32_t px = 0; px < width; ++px) {
      const int64_t pix = (int64_t)py * width + px;
      depth[pix] = INFINITY;
      ijk[3 * pix + 0] = ijk[3 * pix + 1] = ijk[3 * pix + 2] = INT32_MIN;
      label[pix] = -1;
      if (sim) sim[pix] = 0.0;
      float u[3];
      pixel_ray_f32(R, fx, fy, cx, cy, px, py, u);
      vis.clear();
      ray_visits_f32(v, o, u, near_t, far_t, cap, &vis);
      bool have_prev = false;
      double Dp = 0.0, tp = 0.0;
      for (const auto& ii : vis) {
        auto it = m.vox.find(VKey{ii[0], ii[1], ii[2]});
        if (it == m.vox.end()) {
          have_prev = false;
          continue;
        }
        const Rec& r = it->second;
        float e[3];
        for (int a = 0; a < 3; ++a) {
          float fi = (float)ii[a] + 0.5f;
          float c = fi * v;
          e[a] = c - o[a];
        }
        float t0 = e[0] * u[0];
        float t1 = e[1] * u[1];
        float t2 = e[2] * u[2];
        float tc = t0 + t1;
        tc = tc + t2;
        if (have_prev && Dp > 0.0 && r.D <= 0.0) {
          depth[pix] = tp + ((double)tc - tp) * Dp / (Dp - r.D);
          for (int a = 0; a < 3; ++a) ijk[3 * pix + a] = ii[a];
          if (P.mode != OPEN) {
            int best = 0;
            for (int c = 1; c < w; ++c)
              if (r.sem[c] > r.sem[best]) best = c;
            label[pix] = best;
          } else if (q && sim) {
            double dot = 0.0, mn = 0.0;
            for (int c = 0; c < w; ++c) {
              dot += r.sem[c] * (double)q[c];
              mn += r.sem[c] * r.sem[c];
            }
            mn = std::sqrt(mn);
            sim[pix] = (mn > 0.0 && qn > 0.0) ? dot / (mn * qn) : 0.0;
          }
          ++hits;
          break;
        }
        have_prev = true;
        Dp = r.D;
        tp = (double)tc;
      }
    }
  return hits;
}

// Voxels the render ray of one pixel enters (for pinning the traversal).
int64_t ora_pixel_visits(float v, const double world_from_camera[16], float fx, float fy,
                         float cx, float cy, int32_t px, int32_t py, float near_t, float far_t,
                         int32_t* ijk, int64_t cap) {
  float R[9], o[3], u[3];
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) R[a * 3 + b] = (float)world_from_camera[a * 4 + b];
    o[a] = (float)world_from_camera[a * 4 + 3];
  }
  pixel_ray_f32(R, fx, fy, cx, cy, px, py, u);
  std::vector<std::array<int32_t, 3>> vis;
  const int vcap = 3 * (int)std::ceil(((double)far_t - (double)near_t) / (double)v) + 3;
  ray_visits_f32(v, o, u, near_t, far_t, vcap, &vis);
  int64_t k = 0;
  for (auto& a : vis) {
    if (k < cap)
      for (int c = 0; c < 3; ++c) ijk[3 * k + c] = a[c];
    ++k;
  }
  return k;
}

// Open-set read-out (end of Sec. III-D, Fig. "sit"): cosine similarity of each
// voxel mean m (rows, n x l, FP64) against Q query embeddings (Q x l), softmax
// over the queries of cos / temperature, most probable query, kept when its
// probability reaches tp (T_p = 0.1 in the paper), else label -1.
// A zero-norm row gets label -1 and probability 0.
void ora_query(const double* rows, int64_t n, int32_t l, const float* q, int32_t Q,
               double temperature, double tp, int32_t* label, double* prob, double* cosine) {
  std::vector<double> qn((size_t)Q);
  for (int j = 0; j < Q; ++j) {
    double s = 0;
    for (int k = 0; k < l; ++k) s += (double)q[(size_t)j * l + k] * (double)q[(size_t)j * l + k];
    qn[j] = std::sqrt(s);
  }
  std::vector<double> cs((size_t)Q);
  for (int64_t i = 0; i < n; ++i) {
    const double* m = rows + (size_t)i * l;
    double mn = 0;
    for (int k = 0; k < l; ++k) mn += m[k] * m[k];
    mn = std::sqrt(mn);
    if (!(mn > 0)) {
      label[i] = -1;
      prob[i] = 0.0;
      if (cosine)
        for (int j = 0; j < Q; ++j) cosine[(size_t)i * Q + j] = 0.0;
      continue;
    }
    int best = 0;
    for (int j = 0; j < Q; ++j) {
      double dot = 0;
      for (int k = 0; k < l; ++k) dot += m[k] * (double)q[(size_t)j * l + k];
      cs[j] = dot / (mn * qn[j]);
      if (cosine) cosine[(size_t)i * Q + j] = cs[j];
      if (cs[j] > cs[best]) best = j;
    }
    double z = 0;
    for (int j = 0; j < Q; ++j) z += std::exp((cs[j] - cs[best]) / temperature);
    const double pbest = 1.0 / z;
    prob[i] = pbest;
    label[i] = pbest >= tp ? best : -1;
  }
}

// Reverse-mode gradient of a loss L with respect to one scan's inputs, for a
// map with w~ = 1 integrated from empty (so the final state is the batch posterior of all
// observations, Theorems 1-2 with zero priors). Inputs are the loss
// gradients per allocated voxel, in ora_extract order:
//   gD (n_vox), gS (n_vox x w: dL/dc for closed SOFT, dL/dm for open),
//   gB (n_vox x l: dL/dbeta, open set; may be null).
// Outputs for the scan's n points (zero for invalid points):
//   gsem (n x w) and gxyz (n x 3, sensor frame).
// Per observation (v, j) with SDF d = (x - c_v) . u, u = (x - o)/r:
//   D_v = sum d / W_v  ->  dL/dd = gD_v / W_v (0 where d was clamped at tau)
//   dd/dx = u + (I - u u^T)(x - c_v) / r,  x = R p + t  ->  dL/dp = R^T dL/dx
//   closed SOFT: c_v = sum p_j -> dL/dp_j += gS_v
//   open: m_v = sum z / W_v, beta_v = 1/2 sum (z - m_v)^2
//         -> dL/dz_j += gS_v / W_v + gB_v * (z_j - m_v)
// Geometry follows the FP32 path exactly; derivative arithmetic is FP64.
int64_t ora_backward_scan(void* h, const float* pts, int64_t n, const double pose[16],
                          const float* sem, const double* gD, const double* gS,
                          const double* gB, double* gsem, double* gxyz) {
  Map& m = *(Map*)h;
  const Params& P = m.p;
  if (m.order.size() != m.vox.size()) return -1;  // call ora_extract first
  if (P.weighting != 0) return -2;                // the adjoint is for w~ = 1
  std::unordered_map<VKey, int64_t, VKeyHash> index;
  for (size_t j = 0; j < m.order.size(); ++j) index[m.order[j]] = (int64_t)j;
  float R[9], t[3];
  double M[16];
  pose_f32(P, pose, R, t, M);
  const int w = sem_width(P);
  const float v = P.voxel_size, tau = P.trunc;
  std::vector<Pair> pairs;
  for (int64_t j = 0; j < n; ++j) {
    for (int k = 0; k < w; ++k) gsem[j * w + k] = 0.0;
    for (int a = 0; a < 3; ++a) gxyz[j * 3 + a] = 0.0;
    pairs.clear();
    const float* p = pts + 3 * j;
    if (!point_pairs_f32(P, R, t, p, nullptr, &pairs)) continue;
    // the FP32 world point, ray origin and direction the forward pass used
    float x[3];
    for (int a = 0; a < 3; ++a) {
      float m0 = R[a * 3 + 0] * p[0];
      float m1 = R[a * 3 + 1] * p[1];
      float m2 = R[a * 3 + 2] * p[2];
      float s = m0 + m1;
      s = s + m2;
      x[a] = s + t[a];
    }
    double dl[3], xd[3];
    for (int a = 0; a < 3; ++a) {
      xd[a] = (double)x[a];
      dl[a] = xd[a] - (double)t[a];
    }
    const double r = std::sqrt(dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2]);
    double u[3] = {dl[0] / r, dl[1] / r, dl[2] / r};
    double gx[3] = {0, 0, 0};
    const float* s = sem + (size_t)j * w;
    for (const Pair& pr : pairs) {
      VKey key{pr.i[0], pr.i[1], pr.i[2]};
      const int64_t vi = index.at(key);
      const Rec& rec = m.vox.at(key);
      if (P.mode == CLOSED_SOFT) {
        for (int k = 0; k < w; ++k) gsem[j * w + k] += gS[vi * w + k];
      } else if (P.mode == OPEN) {
        for (int k = 0; k < w; ++k) {
          double g = gS[vi * w + k] / rec.W;
          if (gB) g += gB[vi * w + k] * ((double)s[k] - rec.sem[k]);
          gsem[j * w + k] += g;
        }
      }
      if (pr.d >= (double)tau) continue;  // clamped: no dependence on x
      const double gd = gD[vi] / rec.W;
      double e[3], eu = 0;
      for (int a = 0; a < 3; ++a) {
        e[a] = xd[a] - ((double)pr.i[a] + 0.5) * (double)v;
        eu += e[a] * u[a];
      }
      for (int a = 0; a < 3; ++a) gx[a] += gd * (u[a] + (e[a] - u[a] * eu) / r);
    }
    for (int b = 0; b < 3; ++b) {
      double acc = 0;
      for (int a = 0; a < 3; ++a) acc += (double)R[a * 3 + b] * gx[a];
      gxyz[j * 3 + b] = acc;
    }
  }
  return 0;
}

}  // extern "C"
