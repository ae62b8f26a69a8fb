// Host mesh builder: global numbering (the action of Q, Section 3.1), multiplicity
// (Algorithm 1's weights c = 1/multiplicity), Dirichlet mask (Algorithm 1 step 7) and the
// gather-scatter segment lists used by the dssum kernel (Section 4.3).
//
// Numbering rule: two local points are one global node iff they sit on the same
// topological entity at the same position - the same vertex; the same edge (its sorted
// vertex pair) at the same distance from the lower-id end; the same face (its sorted
// vertex 4-set) at the same position in the face frame whose origin is the lowest-id
// corner and whose first axis points to the origin's lower-id neighbour. Global ids are
// assigned in order of first occurrence in the local order (element, k, j, i).
//
// Implementation: edges and faces get ids by sorting their vertex keys; every entity
// position then maps to a dense integer key, and a single pass over the local points
// hands out ids at first sight. Element-interior points are always new.
#include <algorithm>
#include <array>
#include <numeric>

#include "sem_internal.h"

namespace sem {
namespace {

inline int corner(int a, int b, int c) { return a + 2 * b + 4 * c; }

struct ElemFrames {
  int64_t edge_id[12];
  bool edge_rev[12];   // true if the local low end has the larger vertex id
  int64_t face_id[6];
  int8_t face_oa[6], face_ob[6];
  bool face_swap[6];   // true if the canonical first axis is the local second free axis
};

}  // namespace

sem_status build_topology(int N, int64_t nv, int64_t E, const int64_t* ev, const uint8_t* dflags, Topology& T) {
  if (N < 1 || N > SEM_MAX_N) return fail(SEM_ERR_UNSUPPORTED, "polynomial order N must be in [1, SEM_MAX_N]");
  if (E < 1 || nv < 8 || ev == nullptr) return fail(SEM_ERR_ARG, "need E >= 1, num_vertices >= 8 and elem_verts");
  const int Np = N + 1;
  const int64_t P = static_cast<int64_t>(Np) * Np * Np;
  if (E > (int64_t(1) << 31) / P) return fail(SEM_ERR_ARG, "E * (N+1)^3 must be below 2^31");
  const int64_t n = E * P;
  for (int64_t e = 0; e < E; ++e) {
    const int64_t* v = ev + 8 * e;
    for (int a = 0; a < 8; ++a) {
      if (v[a] < 0 || v[a] >= nv) return fail(SEM_ERR_MESH, "element " + std::to_string(e) + ": vertex id out of range");
      for (int b = 0; b < a; ++b)
        if (v[a] == v[b]) return fail(SEM_ERR_MESH, "element " + std::to_string(e) + " repeats a vertex id");
    }
  }

  // ---- edges: local edge d*4 + x + 2y runs along axis d; the other two axes (in order) sit at ends x, y
  std::vector<std::array<int64_t, 2>> ekey(E * 12);
  for (int64_t e = 0; e < E; ++e) {
    const int64_t* v = ev + 8 * e;
    for (int d = 0; d < 3; ++d)
      for (int xy = 0; xy < 4; ++xy) {
        int lo[3], hi[3];
        const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
        lo[d] = 0; hi[d] = 1;
        lo[d1] = hi[d1] = xy & 1;
        lo[d2] = hi[d2] = xy >> 1;
        int64_t a = v[corner(lo[0], lo[1], lo[2])], b = v[corner(hi[0], hi[1], hi[2])];
        ekey[e * 12 + d * 4 + xy] = {std::min(a, b), std::max(a, b)};
      }
  }
  std::vector<int64_t> eorder(E * 12);
  std::iota(eorder.begin(), eorder.end(), 0);
  std::sort(eorder.begin(), eorder.end(), [&](int64_t p, int64_t q) { return ekey[p] < ekey[q]; });
  std::vector<int64_t> edge_of(E * 12);
  int64_t n_edges = 0;
  for (size_t r = 0; r < eorder.size(); ++r) {
    if (r > 0 && ekey[eorder[r]] != ekey[eorder[r - 1]]) ++n_edges;
    edge_of[eorder[r]] = n_edges;
  }
  ++n_edges;
  std::vector<std::array<int64_t, 2>>().swap(ekey);

  // ---- faces: local face d*2 + s has axis d at end s; corners c[a][b] over the other axes (in order)
  std::vector<std::array<int64_t, 4>> fkey(E * 6);
  for (int64_t e = 0; e < E; ++e) {
    const int64_t* v = ev + 8 * e;
    for (int d = 0; d < 3; ++d)
      for (int s = 0; s < 2; ++s) {
        const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
        std::array<int64_t, 4> k4;
        for (int ab = 0; ab < 4; ++ab) {
          int c3[3];
          c3[d] = s; c3[d1] = ab & 1; c3[d2] = ab >> 1;
          k4[ab] = v[corner(c3[0], c3[1], c3[2])];
        }
        std::sort(k4.begin(), k4.end());
        fkey[e * 6 + d * 2 + s] = k4;
      }
  }
  std::vector<int64_t> forder(E * 6);
  std::iota(forder.begin(), forder.end(), 0);
  std::sort(forder.begin(), forder.end(), [&](int64_t p, int64_t q) { return fkey[p] < fkey[q]; });
  std::vector<int64_t> face_of(E * 6);
  std::vector<int32_t> face_count;
  int64_t n_faces = 0;
  for (size_t r = 0; r < forder.size(); ++r) {
    if (r > 0 && fkey[forder[r]] != fkey[forder[r - 1]]) ++n_faces;
    face_of[forder[r]] = n_faces;
    if (static_cast<int64_t>(face_count.size()) <= n_faces) face_count.push_back(0);
    ++face_count[n_faces];
  }
  ++n_faces;
  for (int32_t c : face_count)
    if (c > 2) return fail(SEM_ERR_MESH, "a face is shared by more than two elements");
  std::vector<std::array<int64_t, 4>>().swap(fkey);

  // ---- per-element frames
  auto frames_of = [&](int64_t e) {
    ElemFrames f;
    const int64_t* v = ev + 8 * e;
    for (int d = 0; d < 3; ++d) {
      const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
      for (int xy = 0; xy < 4; ++xy) {
        int lo[3], hi[3];
        lo[d] = 0; hi[d] = 1;
        lo[d1] = hi[d1] = xy & 1;
        lo[d2] = hi[d2] = xy >> 1;
        f.edge_id[d * 4 + xy] = edge_of[e * 12 + d * 4 + xy];
        f.edge_rev[d * 4 + xy] = v[corner(lo[0], lo[1], lo[2])] > v[corner(hi[0], hi[1], hi[2])];
      }
      for (int s = 0; s < 2; ++s) {
        int64_t c[2][2];
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) {
            int c3[3];
            c3[d] = s; c3[d1] = a; c3[d2] = b;
            c[a][b] = v[corner(c3[0], c3[1], c3[2])];
          }
        int oa = 0, ob = 0;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b)
            if (c[a][b] < c[oa][ob]) { oa = a; ob = b; }
        const int lf = d * 2 + s;
        f.face_id[lf] = face_of[e * 6 + lf];
        f.face_oa[lf] = static_cast<int8_t>(oa);
        f.face_ob[lf] = static_cast<int8_t>(ob);
        f.face_swap[lf] = !(c[1 - oa][ob] < c[oa][1 - ob]);
      }
    }
    return f;
  };

  // ---- classification of the P positions of an element (the same for every element)
  struct PosInfo {
    uint8_t cls;     // 0 element interior, 1 vertex, 2 edge, 3 face
    uint8_t idx;     // corner (vertex), local edge (edge), local face (face)
    uint8_t c0, c1;  // coordinate along the edge; the two in-face coordinates
  };
  std::vector<PosInfo> pos(P);
  std::vector<int32_t> bpos;  // element-boundary positions, ascending
  for (int k = 0; k < Np; ++k)
    for (int j = 0; j < Np; ++j)
      for (int i = 0; i < Np; ++i) {
        const int r = (k * Np + j) * Np + i;
        const int q[3] = {i, j, k};
        int end[3], n_end = 0;
        for (int d = 0; d < 3; ++d) {
          end[d] = q[d] == 0 ? 0 : (q[d] == N ? 1 : -1);
          n_end += end[d] >= 0;
        }
        PosInfo pi{0, 0, 0, 0};
        if (n_end == 3) {
          pi = {1, static_cast<uint8_t>(corner(end[0], end[1], end[2])), 0, 0};
        } else if (n_end == 2) {
          const int d = end[0] < 0 ? 0 : (end[1] < 0 ? 1 : 2);
          const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
          pi = {2, static_cast<uint8_t>(d * 4 + end[d1] + 2 * end[d2]), static_cast<uint8_t>(q[d]), 0};
        } else if (n_end == 1) {
          const int d = end[0] >= 0 ? 0 : (end[1] >= 0 ? 1 : 2);
          const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
          pi = {3, static_cast<uint8_t>(d * 2 + end[d]), static_cast<uint8_t>(q[d1]), static_cast<uint8_t>(q[d2])};
        }
        pos[r] = pi;
        if (pi.cls != 0) bpos.push_back(r);
      }

  // ---- numbering, with the copy count of every global node
  const int64_t Nm1 = N - 1;
  const int64_t K_e = nv, K_f = K_e + n_edges * Nm1, n_keys = K_f + n_faces * Nm1 * Nm1;
  std::vector<int32_t> first_id(n_keys, -1);
  std::vector<int32_t> count;
  count.reserve(static_cast<size_t>(n));
  T.glo.assign(n, 0);
  for (int64_t e = 0; e < E; ++e) {
    const ElemFrames f = frames_of(e);
    const int64_t* v = ev + 8 * e;
    int32_t* glo = T.glo.data() + e * P;
    for (int r = 0; r < P; ++r) {
      const PosInfo pi = pos[r];
      int64_t key;
      switch (pi.cls) {
        case 0:  // element interior: always a new node
          glo[r] = static_cast<int32_t>(count.size());
          count.push_back(1);
          continue;
        case 1:
          key = v[pi.idx];
          break;
        case 2: {
          const int t = f.edge_rev[pi.idx] ? N - pi.c0 : pi.c0;
          key = K_e + f.edge_id[pi.idx] * Nm1 + (t - 1);
          break;
        }
        default: {
          const int lf = pi.idx;
          const int ps = f.face_oa[lf] == 0 ? pi.c0 : N - pi.c0;
          const int pt = f.face_ob[lf] == 0 ? pi.c1 : N - pi.c1;
          const int p0 = f.face_swap[lf] ? pt : ps, p1 = f.face_swap[lf] ? ps : pt;
          key = K_f + f.face_id[lf] * Nm1 * Nm1 + (p0 - 1) * Nm1 + (p1 - 1);
          break;
        }
      }
      int32_t& g = first_id[key];
      if (g < 0) {
        g = static_cast<int32_t>(count.size());
        count.push_back(0);
      }
      ++count[g];
      glo[r] = g;
    }
  }
  std::vector<int32_t>().swap(first_id);
  const int64_t n_glob = static_cast<int64_t>(count.size());

  // ---- multiplicity (element-interior copies have multiplicity 1)
  T.mult.assign(n, 1);
  for (int64_t e = 0; e < E; ++e)
    for (const int32_t r : bpos) {
      const int32_t c = count[T.glo[e * P + r]];
      if (c > 255) return fail(SEM_ERR_MESH, "a global node has more than 255 local copies");
      T.mult[e * P + r] = static_cast<uint8_t>(c);
    }

  // ---- Dirichlet mask: points on the closure of a boundary face (owned by one element)
  std::vector<uint8_t> mglob(n_glob, 0);
  for (int64_t e = 0; e < E; ++e) {
    const int64_t* v = ev + 8 * e;
    for (int d = 0; d < 3; ++d)
      for (int s = 0; s < 2; ++s) {
        const int lf = d * 2 + s;
        if (face_count[face_of[e * 6 + lf]] != 1) continue;
        if (dflags) {
          const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
          bool all = true;
          for (int ab = 0; ab < 4; ++ab) {
            int c3[3];
            c3[d] = s; c3[d1] = ab & 1; c3[d2] = ab >> 1;
            all = all && dflags[v[corner(c3[0], c3[1], c3[2])]] != 0;
          }
          if (!all) continue;
        }
        for (const int32_t r : bpos) {
          const int q[3] = {r % Np, (r / Np) % Np, r / (Np * Np)};
          if (q[d] == s * N) mglob[T.glo[e * P + r]] = 1;
        }
      }
  }
  T.mask.assign(n, 0);  // element-interior points are never on a boundary face
  for (int64_t e = 0; e < E; ++e)
    for (const int32_t r : bpos) T.mask[e * P + r] = mglob[T.glo[e * P + r]];

  // ---- gather-scatter segments: global nodes with copies on element boundaries, ascending
  // id; a boundary node's copies all lie on element boundaries, so its copy count is its size
  std::vector<int32_t> seg_of(n_glob, -1);
  std::vector<uint8_t> is_bdry(n_glob, 0);
  for (int64_t e = 0; e < E; ++e)
    for (const int32_t r : bpos) is_bdry[T.glo[e * P + r]] = 1;
  T.seg_off.clear();
  T.seg_off.push_back(0);
  T.seg_mask.clear();
  for (int64_t g = 0; g < n_glob; ++g)
    if (is_bdry[g]) {
      seg_of[g] = static_cast<int32_t>(T.seg_off.size() - 1);
      T.seg_off.push_back(T.seg_off.back() + count[g]);
      T.seg_mask.push_back(mglob[g]);
    }
  std::vector<int32_t> cursor(T.seg_off.begin(), T.seg_off.end() - 1);
  T.seg_idx.assign(T.seg_off.back(), 0);
  for (int64_t e = 0; e < E; ++e)
    for (const int32_t r : bpos) {
      const int64_t loc = e * P + r;
      T.seg_idx[cursor[seg_of[T.glo[loc]]]++] = static_cast<int32_t>(loc);
    }

  T.N = N;
  T.Np = Np;
  T.E = E;
  T.n = n;
  T.n_glob = n_glob;
  return SEM_OK;
}

}  // namespace sem
