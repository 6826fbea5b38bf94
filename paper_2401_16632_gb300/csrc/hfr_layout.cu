// Host-side trace layouts that do not need a device: the node numbering of the interior-embedded
// (EFR) trace space (Sec. 2.2: trace continuous on the implicit skeleton, nodes at the
// Gauss-Lobatto points of every trace face, vertices shared by the faces that meet there).
//
// Vertices are found by union-find over element corners: the two ends of a trace face are joined
// to the matching ends of the neighbour's face (all elements share one orientation, so the first
// point of a face meets the first point of the neighbour's).  Each class is named by its smallest
// corner index 4 e + c; vertex nodes are numbered in increasing name, then the p - 1 interior
// points of trace face t (trace faces in increasing global face id) at nvert + t (p - 1) + m - 1.

#include <algorithm>
#include <vector>

#include "../../include/hfr.h"

namespace {

// corners (a + 2 b) at the first and the last point of local faces 0..3
constexpr int kFaceCorner[4][2] = {{0, 2}, {1, 3}, {0, 1}, {2, 3}};

int find_root(std::vector<int>& parent, int i) {
  while (parent[i] != i) {
    parent[i] = parent[parent[i]];
    i = parent[i];
  }
  return i;
}

}  // namespace

static int efr_trace_nodes_impl(int nelem, const int* nbr, const int* nbr_face, const int* face_of, const int* bc,
                                const unsigned char* implicit, int p, int* node_of, int* nvert_out, int* nnode_out) {
  if (nelem <= 0 || !nbr || !nbr_face || !face_of || !implicit || !node_of || !nvert_out || !nnode_out)
    return FR_ERR_INVALID_ARG;
  if (p < 1 || p > 5) return FR_ERR_INVALID_ARG;
  const int n = p + 1;
  int nface = 0;
  for (int e = 0; e < nelem; ++e) {
    for (int f = 0; f < 4; ++f) {
      const int nb = nbr[4 * e + f], nf = nbr_face[4 * e + f], id = face_of[4 * e + f];
      if (id < 0 || (long long)id >= 4LL * nelem) return FR_ERR_INVALID_ARG;
      nface = std::max(nface, id + 1);
      if (nb < 0) {  // boundary face: wall or far field
        if (!bc) return FR_ERR_UNSUPPORTED;
        if (bc[4 * e + f] != 1 && bc[4 * e + f] != 2) return FR_ERR_INVALID_ARG;
        continue;
      }
      if (nb >= nelem || nf < 0 || nf > 3) return FR_ERR_INVALID_ARG;
      if (nbr[4 * nb + nf] != e || nbr_face[4 * nb + nf] != f || face_of[4 * nb + nf] != id)
        return FR_ERR_INVALID_ARG;  // the neighbour relation must be symmetric
    }
  }
  // trace faces: both sides implicit, numbered in increasing global face id; boundary faces of
  // implicit elements (discontinuous traces at their Gauss points) numbered apart, the same way
  std::vector<int> trace_of_face(nface, -1), bface_of(nface, -1);
  for (int e = 0; e < nelem; ++e)
    for (int f = 0; f < 4; ++f) {
      const int nb = nbr[4 * e + f];
      if (nb >= 0 && implicit[e] && implicit[nb]) trace_of_face[face_of[4 * e + f]] = 0;
      if (nb < 0 && implicit[e]) bface_of[face_of[4 * e + f]] = 0;
    }
  int nbface = 0;
  for (int id = 0; id < nface; ++id)
    if (bface_of[id] == 0) bface_of[id] = nbface++;
  int ntrace = 0;
  for (int id = 0; id < nface; ++id)
    if (trace_of_face[id] == 0) trace_of_face[id] = ntrace++;
  // vertex classes over element corners, joined through trace faces only
  std::vector<int> parent(4 * static_cast<size_t>(nelem));
  for (size_t i = 0; i < parent.size(); ++i) parent[i] = static_cast<int>(i);
  std::vector<unsigned char> touched(parent.size(), 0);
  for (int e = 0; e < nelem; ++e) {
    if (!implicit[e]) continue;
    for (int f = 0; f < 4; ++f) {
      const int nb = nbr[4 * e + f], nf = nbr_face[4 * e + f];
      if (nb < 0 || !implicit[nb]) continue;
      for (int end = 0; end < 2; ++end) {
        const int i = 4 * e + kFaceCorner[f][end], j = 4 * nb + kFaceCorner[nf][end];
        touched[i] = touched[j] = 1;
        const int ri = find_root(parent, i), rj = find_root(parent, j);
        if (ri != rj) parent[std::max(ri, rj)] = std::min(ri, rj);
      }
    }
  }
  std::vector<int> vertex_id(parent.size(), -1);
  int nvert = 0;
  for (size_t i = 0; i < parent.size(); ++i)  // roots are the smallest corners of their classes
    if (touched[i] && find_root(parent, static_cast<int>(i)) == static_cast<int>(i)) vertex_id[i] = nvert++;
  for (int e = 0; e < nelem; ++e) {
    for (int f = 0; f < 4; ++f) {
      int* out = node_of + (static_cast<size_t>(e) * 4 + f) * n;
      const int nb = nbr[4 * e + f];
      if (nb < 0 && implicit[e]) {  // boundary trace: n nodes of its own after the interior ones
        const int base = nvert + ntrace * (n - 2) + bface_of[face_of[4 * e + f]] * n;
        for (int m = 0; m < n; ++m) out[m] = base + m;
        continue;
      }
      if (!implicit[e] || nb < 0 || !implicit[nb]) {
        std::fill(out, out + n, -1);
        continue;
      }
      const int t = trace_of_face[face_of[4 * e + f]];
      out[0] = vertex_id[find_root(parent, 4 * e + kFaceCorner[f][0])];
      out[n - 1] = vertex_id[find_root(parent, 4 * e + kFaceCorner[f][1])];
      for (int m = 1; m < n - 1; ++m) out[m] = nvert + t * (n - 2) + m - 1;
    }
  }
  *nvert_out = nvert;
  *nnode_out = nvert + ntrace * (n - 2) + nbface * n;
  return FR_OK;
}

// Trace layout of a mesh whose elements carry different degrees (faces between unequal degrees
// carry the Gauss points of the higher one; boundary faces the element's own), with wall and
// far-field faces: a face has a trace when both sides are implicit, or when it is a boundary face
// of an implicit element; traces are numbered in increasing global face id and stored one after
// the other, trace t holding face_pts points from trace_off[t].
static int mixed_trace_layout_impl(int nelem, const int* nbr, const int* nbr_face, const int* face_of, const int* bc,
                                  const unsigned char* implicit, const int* p, int* face_pts, int* trace_of,
                                  int* trace_off, int* ntrace_out) {
  if (nelem <= 0 || !nbr || !nbr_face || !face_of || !bc || !implicit || !p || !face_pts || !trace_of ||
      !trace_off || !ntrace_out)
    return FR_ERR_INVALID_ARG;
  int nface = 0;
  for (int e = 0; e < nelem; ++e) {
    if (p[e] < 1 || p[e] > 5) return FR_ERR_INVALID_ARG;
    for (int f = 0; f < 4; ++f) {
      const int nb = nbr[4 * e + f], nf = nbr_face[4 * e + f], id = face_of[4 * e + f];
      if (id < 0 || (long long)id >= 4LL * nelem) return FR_ERR_INVALID_ARG;  // at most 4 nelem faces
      nface = std::max(nface, id + 1);
      if (nb < 0) {
        if (bc[4 * e + f] != 1 && bc[4 * e + f] != 2) return FR_ERR_INVALID_ARG;  // wall or far field
        continue;
      }
      if (nb >= nelem || nf < 0 || nf > 3) return FR_ERR_INVALID_ARG;
      if (nbr[4 * nb + nf] != e || nbr_face[4 * nb + nf] != f || face_of[4 * nb + nf] != id)
        return FR_ERR_INVALID_ARG;
    }
  }
  std::vector<int> trace_of_face(nface, -1), pts_of_face(nface, 0);
  for (int e = 0; e < nelem; ++e) {
    for (int f = 0; f < 4; ++f) {
      const int nb = nbr[4 * e + f];
      const int pts = (nb < 0 ? p[e] : std::max(p[e], p[nb])) + 1;
      face_pts[4 * e + f] = pts;
      const bool traced = implicit[e] && (nb < 0 || implicit[nb]);
      if (traced) {
        trace_of_face[face_of[4 * e + f]] = 0;
        pts_of_face[face_of[4 * e + f]] = pts;
      }
    }
  }
  int ntrace = 0;
  trace_off[0] = 0;
  for (int id = 0; id < nface; ++id) {
    if (trace_of_face[id] != 0) continue;
    trace_of_face[id] = ntrace;
    trace_off[ntrace + 1] = trace_off[ntrace] + pts_of_face[id];
    ++ntrace;
  }
  for (int e = 0; e < nelem; ++e)
    for (int f = 0; f < 4; ++f) {
      const int nb = nbr[4 * e + f];
      trace_of[4 * e + f] = (implicit[e] && (nb < 0 || implicit[nb])) ? trace_of_face[face_of[4 * e + f]] : -1;
    }
  *ntrace_out = ntrace;
  return FR_OK;
}

// the host vectors may fail to allocate: no C++ exception crosses the C ABI
extern "C" int efr_trace_nodes(int nelem, const int* nbr, const int* nbr_face, const int* face_of, const int* bc,
                               const unsigned char* implicit, int p, int* node_of, int* nvert_out,
                               int* nnode_out) {
  try {
    return efr_trace_nodes_impl(nelem, nbr, nbr_face, face_of, bc, implicit, p, node_of, nvert_out, nnode_out);
  } catch (...) {
    return FR_ERR_OOM;
  }
}

extern "C" int mixed_trace_layout(int nelem, const int* nbr, const int* nbr_face, const int* face_of, const int* bc,
                                  const unsigned char* implicit, const int* p, int* face_pts, int* trace_of,
                                  int* trace_off, int* ntrace_out) {
  try {
    return mixed_trace_layout_impl(nelem, nbr, nbr_face, face_of, bc, implicit, p, face_pts, trace_of, trace_off,
                                   ntrace_out);
  } catch (...) {
    return FR_ERR_OOM;
  }
}
