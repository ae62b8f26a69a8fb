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
// Implementation: edges and faces get ids by sorting their vertex keys (ties by position, so
// every entity lists the elements that hold it in ascending order); each vertex, edge and
// face knows the first element that holds it, how many elements hold it and whether it lies
// on a Dirichlet face. A node is new in element e iff its entity's first element is e, so
// the count of new nodes per element, a prefix sum over elements and two passes over the
// elements (new nodes, then the nodes seen before) number every point; these passes, the
// multiplicities, the mask and the segment lists run on all host threads, element by
// element, and give the same result as a sequential pass. Element-interior points are
// always new.
#include <algorithm>
#include <array>
#include <memory>
#include <numeric>
#include <thread>

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

// Calls f(begin, end) on contiguous chunks of [0, n), one per host thread (at most 32, and
// chunks of at least `grain` items); the calling thread takes the first chunk. f must not
// throw. If a thread cannot be started its chunk runs on the calling thread.
template <typename F>
void parallel_for(int64_t n, int64_t grain, const F& f) {
  if (n <= 0) return;
  const unsigned hw = std::thread::hardware_concurrency();
  int64_t T = hw == 0 ? 1 : std::min<int64_t>(hw, 32);
  T = std::max<int64_t>(1, std::min<int64_t>(T, (n + grain - 1) / grain));
  const int64_t chunk = (n + T - 1) / T;
  std::vector<std::thread> th;
  th.reserve(static_cast<size_t>(T));
  for (int64_t t = 1; t < T; ++t) {
    const int64_t b = t * chunk, e = std::min(n, b + chunk);
    if (b >= e) break;
    try {
      th.emplace_back([&f, b, e] { f(b, e); });
    } catch (...) {
      f(b, e);
    }
  }
  f(int64_t(0), std::min(n, chunk));
  for (auto& x : th) x.join();
}

// Sorts records whose first key is a vertex id in [0, nv) lexicographically: a stable counting
// sort by the first key, then each (small) bucket sorted by the remaining keys on all host
// threads. With distinct records the result is that of std::sort.
template <size_t K>
void sort_by_vertex(std::vector<std::array<int64_t, K>>& rec, int64_t nv) {
  std::vector<int64_t> start(static_cast<size_t>(nv) + 1, 0);
  for (const auto& x : rec) ++start[x[0] + 1];
  for (int64_t v = 0; v < nv; ++v) start[v + 1] += start[v];
  std::vector<std::array<int64_t, K>> out(rec.size());
  {
    std::vector<int64_t> at(start.begin(), start.end() - 1);
    for (const auto& x : rec) out[at[x[0]]++] = x;
  }
  parallel_for(nv, 4096, [&](int64_t v0, int64_t v1) {
    for (int64_t v = v0; v < v1; ++v) std::sort(out.begin() + start[v], out.begin() + start[v + 1]);
  });
  rec.swap(out);
}

// Entity of an element-boundary position: dense key of the node, first element holding the
// entity, number of elements holding it, Dirichlet flag, rank of this element among them.
struct PosEntity {
  int64_t key;
  int64_t first;
  int32_t count;
  uint8_t dir;
  int32_t rank;
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
  constexpr int64_t kGrain = 256;  // elements per chunk at least

  // ---- vertices: the elements holding each vertex, ascending, and each element's rank
  std::vector<int32_t> vcount(nv, 0);
  for (int64_t q = 0; q < 8 * E; ++q) ++vcount[ev[q]];
  for (int64_t x = 0; x < nv; ++x)
    if (vcount[x] > 255) return fail(SEM_ERR_MESH, "a global node has more than 255 local copies");
  std::vector<int64_t> vfirst(nv, -1);
  std::vector<int32_t> vseen(nv, 0);
  std::vector<uint8_t> vrank(8 * E);
  for (int64_t q = 0; q < 8 * E; ++q) {
    const int64_t x = ev[q];
    if (vfirst[x] < 0) vfirst[x] = q / 8;
    vrank[q] = static_cast<uint8_t>(vseen[x]++);
  }
  std::vector<int32_t>().swap(vseen);

  // ---- edges: local edge d*4 + x + 2y runs along axis d; the other two axes (in order) sit at ends x, y.
  // Records (low vertex, high vertex, position e*12 + edge) sorted; ties by position.
  std::vector<std::array<int64_t, 3>> erec(E * 12);
  parallel_for(E, kGrain, [&](int64_t b0, int64_t b1) {
    for (int64_t e = b0; e < b1; ++e) {
      const int64_t* v = ev + 8 * e;
      for (int d = 0; d < 3; ++d)
        for (int xy = 0; xy < 4; ++xy) {
          int lo[3], hi[3];
          const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
          lo[d] = 0; hi[d] = 1;
          lo[d1] = hi[d1] = xy & 1;
          lo[d2] = hi[d2] = xy >> 1;
          const int64_t a = v[corner(lo[0], lo[1], lo[2])], c = v[corner(hi[0], hi[1], hi[2])];
          erec[e * 12 + d * 4 + xy] = {std::min(a, c), std::max(a, c), e * 12 + d * 4 + xy};
        }
    }
  });
  // ---- faces: local face d*2 + s has axis d at end s; corners c[a][b] over the other axes (in order).
  // Records (sorted four vertex ids, position e*6 + face) sorted; ties by position.
  std::vector<std::array<int64_t, 5>> frec(E * 6);
  parallel_for(E, kGrain, [&](int64_t b0, int64_t b1) {
    for (int64_t e = b0; e < b1; ++e) {
      const int64_t* v = ev + 8 * e;
      for (int d = 0; d < 3; ++d)
        for (int s = 0; s < 2; ++s) {
          const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
          std::array<int64_t, 5> k5;
          for (int ab = 0; ab < 4; ++ab) {
            int c3[3];
            c3[d] = s; c3[d1] = ab & 1; c3[d2] = ab >> 1;
            k5[ab] = v[corner(c3[0], c3[1], c3[2])];
          }
          std::sort(k5.begin(), k5.begin() + 4);
          k5[4] = e * 6 + d * 2 + s;
          frec[e * 6 + d * 2 + s] = k5;
        }
    }
  });
  sort_by_vertex(erec, nv);
  sort_by_vertex(frec, nv);
  std::vector<int64_t> edge_of(E * 12), efirst;
  std::vector<int32_t> ecount;
  efirst.reserve(E * 12);
  ecount.reserve(E * 12);
  std::vector<uint8_t> erank(E * 12);
  for (size_t r = 0; r < erec.size(); ++r) {
    if (r == 0 || erec[r][0] != erec[r - 1][0] || erec[r][1] != erec[r - 1][1]) {
      efirst.push_back(erec[r][2] / 12);
      ecount.push_back(0);
    }
    edge_of[erec[r][2]] = static_cast<int64_t>(efirst.size()) - 1;
    if (ecount.back() >= 255) return fail(SEM_ERR_MESH, "a global node has more than 255 local copies");
    erank[erec[r][2]] = static_cast<uint8_t>(ecount.back()++);
  }
  const int64_t n_edges = static_cast<int64_t>(efirst.size());
  std::vector<std::array<int64_t, 3>>().swap(erec);
  std::vector<int64_t> face_of(E * 6), ffirst;
  std::vector<int32_t> face_count;
  ffirst.reserve(E * 6);
  face_count.reserve(E * 6);
  std::vector<uint8_t> frank(E * 6);
  for (size_t r = 0; r < frec.size(); ++r) {
    if (r == 0 || !std::equal(frec[r].begin(), frec[r].begin() + 4, frec[r - 1].begin())) {
      ffirst.push_back(frec[r][4] / 6);
      face_count.push_back(0);
    }
    face_of[frec[r][4]] = static_cast<int64_t>(ffirst.size()) - 1;
    frank[frec[r][4]] = static_cast<uint8_t>(face_count.back()++);
    if (face_count.back() > 2) return fail(SEM_ERR_MESH, "a face is shared by more than two elements");
  }
  const int64_t n_faces = static_cast<int64_t>(ffirst.size());
  std::vector<std::array<int64_t, 5>>().swap(frec);

  // ---- per-element frames
  std::vector<ElemFrames> frames(E);
  parallel_for(E, kGrain, [&](int64_t b0, int64_t b1) {
    for (int64_t e = b0; e < b1; ++e) {
      ElemFrames& f = frames[e];
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
    }
  });
  std::vector<int64_t>().swap(edge_of);
  std::vector<int64_t>().swap(face_of);

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

  // ---- Dirichlet entities: boundary faces (owned by one element; with vertex flags, only
  // those whose four vertices are flagged) and the edges and vertices of their closure.
  // The corners and edges on local face d*2 + s, from the position classification.
  std::vector<int> lf_corners[6], lf_edges[6];
  for (int d = 0; d < 3; ++d)
    for (int s = 0; s < 2; ++s)
      for (const int32_t r : bpos) {
        const int q[3] = {r % Np, (r / Np) % Np, r / (Np * Np)};
        if (q[d] != s * N) continue;
        std::vector<int>& list = pos[r].cls == 1 ? lf_corners[d * 2 + s] : lf_edges[d * 2 + s];
        if ((pos[r].cls == 1 || pos[r].cls == 2) && std::find(list.begin(), list.end(), pos[r].idx) == list.end())
          list.push_back(pos[r].idx);
      }
  std::vector<uint8_t> fdir(n_faces, 0), edir(n_edges, 0), vdir(nv, 0);
  for (int64_t e = 0; e < E; ++e) {
    const int64_t* v = ev + 8 * e;
    const ElemFrames& f = frames[e];
    for (int d = 0; d < 3; ++d)
      for (int s = 0; s < 2; ++s) {
        const int lf = d * 2 + s;
        if (face_count[f.face_id[lf]] != 1) continue;
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
        fdir[f.face_id[lf]] = 1;
        for (const int c : lf_corners[lf]) vdir[v[c]] = 1;
        for (const int le : lf_edges[lf]) edir[f.edge_id[le]] = 1;
      }
  }

  // ---- the entity of a boundary position of element e
  const int64_t Nm1 = N - 1;
  const int64_t K_e = nv, K_f = K_e + n_edges * Nm1, n_keys = K_f + n_faces * Nm1 * Nm1;
  // (the tables are captured as plain pointers: the byte-wide stores of the passes below may
  // alias anything, and pointers held in the closure need not be reloaded after them)
  auto entity = [ev, N, Nm1, K_e, K_f, vf = vfirst.data(), vc = vcount.data(), vd = vdir.data(),
                 vr = vrank.data(), ef = efirst.data(), ec = ecount.data(), ed = edir.data(), er = erank.data(),
                 ff = ffirst.data(), fc = face_count.data(), fd = fdir.data(),
                 fr = frank.data()](int64_t e, const ElemFrames& f, const PosInfo& pi) -> PosEntity {
    const int64_t* v = ev + 8 * e;
    if (pi.cls == 1) {
      const int64_t x = v[pi.idx];
      return {x, vf[x], vc[x], vd[x], vr[8 * e + pi.idx]};
    }
    if (pi.cls == 2) {
      const int64_t id = f.edge_id[pi.idx];
      const int t = f.edge_rev[pi.idx] ? N - pi.c0 : pi.c0;
      return {K_e + id * Nm1 + (t - 1), ef[id], ec[id], ed[id], er[12 * e + pi.idx]};
    }
    const int lf = pi.idx;
    const int64_t id = f.face_id[lf];
    const int ps = f.face_oa[lf] == 0 ? pi.c0 : N - pi.c0;
    const int pt = f.face_ob[lf] == 0 ? pi.c1 : N - pi.c1;
    const int p0 = f.face_swap[lf] ? pt : ps, p1 = f.face_swap[lf] ? ps : pt;
    return {K_f + id * Nm1 * Nm1 + (p0 - 1) * Nm1 + (p1 - 1), ff[id], fc[id], fd[id], fr[6 * e + lf]};
  };

  // ---- new nodes per element and the first id of each element's new nodes (prefix sum)
  const int64_t n_int = Nm1 * Nm1 * Nm1;
  std::vector<int64_t> base(E + 1, 0);
  parallel_for(E, kGrain, [&](int64_t b0, int64_t b1) {
    for (int64_t e = b0; e < b1; ++e) {
      const int64_t* v = ev + 8 * e;
      const ElemFrames& f = frames[e];
      int64_t c = n_int;
      for (int a = 0; a < 8; ++a) c += vfirst[v[a]] == e;
      for (int le = 0; le < 12; ++le) c += efirst[f.edge_id[le]] == e ? Nm1 : 0;
      for (int lf = 0; lf < 6; ++lf) c += ffirst[f.face_id[lf]] == e ? Nm1 * Nm1 : 0;
      base[e + 1] = c;
    }
  });
  for (int64_t e = 0; e < E; ++e) base[e + 1] += base[e];
  const int64_t n_glob = base[E];

  // ---- ids of the new nodes of each element (the others get theirs in the segment pass)
  std::unique_ptr<int32_t[]> first_id(new int32_t[n_keys]);
  std::unique_ptr<uint8_t[]> gcount(new uint8_t[n_glob]);  // copies of a boundary node, 0 if interior
  std::unique_ptr<uint8_t[]> gdir(new uint8_t[n_glob]);
  T.glo.resize(n);  // every element written below
  T.mult.resize(n);
  T.mask.resize(n);
  parallel_for(E, kGrain, [&](int64_t b0, int64_t b1) {
    const PosInfo* const ps = pos.data();
    const ElemFrames* const fr = frames.data();
    int32_t* __restrict__ const fid = first_id.get();
    uint8_t* __restrict__ const gc = gcount.get();
    uint8_t* __restrict__ const gd = gdir.get();
    for (int64_t e = b0; e < b1; ++e) {
      const ElemFrames& f = fr[e];
      int32_t* __restrict__ const glo = T.glo.data() + e * P;
      uint8_t* __restrict__ const mult = T.mult.data() + e * P;
      uint8_t* __restrict__ const mask = T.mask.data() + e * P;
      int64_t id = base[e];
      for (int r = 0; r < P; ++r) {
        const PosInfo pi = ps[r];
        if (pi.cls == 0) {  // element interior: a new node, one copy, never on a boundary face
          gc[id] = 0;
          gd[id] = 0;
          mult[r] = 1;
          mask[r] = 0;
          glo[r] = static_cast<int32_t>(id++);
          continue;
        }
        const PosEntity pe = entity(e, f, pi);
        mult[r] = static_cast<uint8_t>(pe.count);
        mask[r] = pe.dir;
        if (pe.first == e) {
          fid[pe.key] = static_cast<int32_t>(id);
          gc[id] = static_cast<uint8_t>(pe.count);
          gd[id] = pe.dir;
          glo[r] = static_cast<int32_t>(id++);
        }
      }
    }
  });

  // ---- gather-scatter segments: boundary nodes in ascending id (chunked prefix sums over
  // the global ids); the copies of a node sit in the ascending list of the elements that hold
  // its entity, so a copy's slot is its segment's start plus its element's rank in that list.
  // The last pass also gives the element-boundary points first seen in earlier elements
  // their ids.
  HostVec<int32_t> seg_of;
  seg_of.resize(n_glob);  // every element written below
  const int64_t gchunk = int64_t(1) << 16, n_gch = (n_glob + gchunk - 1) / gchunk;
  std::vector<int64_t> ch_seg(n_gch + 1, 0), ch_cp(n_gch + 1, 0);
  parallel_for(n_gch, 1, [&](int64_t c0, int64_t c1) {
    for (int64_t c = c0; c < c1; ++c) {
      int64_t s = 0, cp = 0;
      for (int64_t g = c * gchunk; g < std::min(n_glob, (c + 1) * gchunk); ++g) {
        s += gcount[g] > 0;
        cp += gcount[g];
      }
      ch_seg[c + 1] = s;
      ch_cp[c + 1] = cp;
    }
  });
  for (int64_t c = 0; c < n_gch; ++c) {
    ch_seg[c + 1] += ch_seg[c];
    ch_cp[c + 1] += ch_cp[c];
  }
  const int64_t S = ch_seg[n_gch];
  T.seg_off.resize(S + 1);  // every element written below
  T.seg_mask.resize(S);
  T.seg_off[S] = static_cast<int32_t>(ch_cp[n_gch]);
  parallel_for(n_gch, 1, [&](int64_t c0, int64_t c1) {
    for (int64_t c = c0; c < c1; ++c) {
      int64_t s = ch_seg[c], cp = ch_cp[c];
      for (int64_t g = c * gchunk; g < std::min(n_glob, (c + 1) * gchunk); ++g) {
        if (gcount[g] == 0) {
          seg_of[g] = -1;
          continue;
        }
        seg_of[g] = static_cast<int32_t>(s);
        T.seg_off[s] = static_cast<int32_t>(cp);
        T.seg_mask[s] = gdir[g];
        ++s;
        cp += gcount[g];
      }
    }
  });
  T.seg_idx.resize(T.seg_off[S]);  // every slot written once below
  parallel_for(E, kGrain, [&](int64_t b0, int64_t b1) {
    const PosInfo* const ps = pos.data();
    const ElemFrames* const fr = frames.data();
    const int32_t* const fid = first_id.get();
    const int32_t* const so = seg_of.data();
    const int32_t* const off = T.seg_off.data();
    int32_t* __restrict__ const idx = T.seg_idx.data();
    const int32_t* const bp = bpos.data();
    const int64_t nb = static_cast<int64_t>(bpos.size());
    for (int64_t e = b0; e < b1; ++e) {
      const ElemFrames& f = fr[e];
      int32_t* __restrict__ const glo = T.glo.data() + e * P;
      for (int64_t q = 0; q < nb; ++q) {
        const int32_t r = bp[q];
        const PosEntity pe = entity(e, f, ps[r]);
        if (pe.first != e) glo[r] = fid[pe.key];
        idx[off[so[glo[r]]] + pe.rank] = static_cast<int32_t>(e * P + r);
      }
    }
  });
  first_id.reset();

  T.N = N;
  T.Np = Np;
  T.E = E;
  T.n = n;
  T.n_glob = n_glob;
  return SEM_OK;
}

void build_gs_host(const Topology& T, GsHost& H) {
  static constexpr int kW[4] = {1, 2, 4, 8};
  const int64_t S = static_cast<int64_t>(T.seg_mask.size());
  auto cls = [](int c) { return c <= 1 ? 0 : c <= 2 ? 1 : c <= 4 ? 2 : c <= 8 ? 3 : 4; };
  // per chunk of segments: how many fall in each class (and copies of the CSR class)
  const int64_t chunk = int64_t(1) << 15, n_ch = (S + chunk - 1) / chunk;
  std::vector<std::array<int64_t, 6>> cnt(n_ch + 1, std::array<int64_t, 6>{0, 0, 0, 0, 0, 0});
  parallel_for(n_ch, 1, [&](int64_t c0, int64_t c1) {
    for (int64_t c = c0; c < c1; ++c) {
      std::array<int64_t, 6> k{0, 0, 0, 0, 0, 0};
      for (int64_t s = c * chunk; s < std::min(S, (c + 1) * chunk); ++s) {
        const int n = T.seg_off[s + 1] - T.seg_off[s];
        ++k[cls(n)];
        if (cls(n) == 4) k[5] += n;
      }
      cnt[c + 1] = k;
    }
  });
  for (int64_t c = 0; c < n_ch; ++c)
    for (int q = 0; q < 6; ++q) cnt[c + 1][q] += cnt[c][q];
  for (int q = 0; q < 4; ++q) {
    H.rec[q].resize(cnt[n_ch][q] * kW[q]);
    H.msk[q].resize(cnt[n_ch][q]);
  }
  H.xoff.resize(cnt[n_ch][4] + 1);
  H.xidx.resize(cnt[n_ch][5]);
  H.xmsk.resize(cnt[n_ch][4]);
  H.xoff[cnt[n_ch][4]] = static_cast<int32_t>(cnt[n_ch][5]);
  parallel_for(n_ch, 1, [&](int64_t c0, int64_t c1) {
    for (int64_t c = c0; c < c1; ++c) {
      std::array<int64_t, 6> at = cnt[c];
      for (int64_t s = c * chunk; s < std::min(S, (c + 1) * chunk); ++s) {
        const int o0 = T.seg_off[s], n = T.seg_off[s + 1] - o0, q = cls(n);
        if (q < 4) {
          int32_t* r = H.rec[q].data() + at[q] * kW[q];
          for (int k = 0; k < kW[q]; ++k) r[k] = k < n ? T.seg_idx[o0 + k] : -1;
          H.msk[q][at[q]++] = T.seg_mask[s];
        } else {
          H.xoff[at[4]] = static_cast<int32_t>(at[5]);
          for (int k = 0; k < n; ++k) H.xidx[at[5]++] = T.seg_idx[o0 + k];
          H.xmsk[at[4]++] = T.seg_mask[s];
        }
      }
    }
  });
}

}  // namespace sem
