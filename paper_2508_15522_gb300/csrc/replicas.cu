// Replica sets: molecule templates (per-atom parameters of Sec. 3, the
// reduced UFF-like topology), replica-major state arrays, state I/O.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"
#include "trace.h"

namespace {

template <class T>
size_t push(std::vector<unsigned char>& blob, const std::vector<T>& v) {
  size_t off = (blob.size() + 255) & ~size_t(255);
  blob.resize(off + v.size() * sizeof(T));
  if (!v.empty()) memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
  return off;
}

bool copy_in(gridff_ctx* ctx, void* dst, const void* src, size_t bytes, int flags) {
  cudaMemcpyKind k = (flags & GRIDFF_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  return cudaMemcpyAsync(dst, src, bytes, k, ctx->stream) == cudaSuccess;
}

bool copy_out(gridff_ctx* ctx, void* dst, const void* src, size_t bytes, int flags) {
  cudaMemcpyKind k = (flags & GRIDFF_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  return cudaMemcpyAsync(dst, src, bytes, k, ctx->stream) == cudaSuccess;
}

gridff_status finish(gridff_ctx* ctx, int flags) {
  if ((flags & GRIDFF_ASYNC) && (flags & GRIDFF_DEVICE_PTRS)) return GRIDFF_OK;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return set_err(ctx, GRIDFF_ECUDA, "%s", cudaGetErrorString(e));
  return GRIDFF_OK;
}

// Order of the unique bonded terms of a template: the kernels give 32
// consecutive terms to the 32 lanes of a warp, and each term adds its
// forces to s_f[3 atom + comp] with one shared-memory atomic per role and
// component.  Lanes whose atoms of a role fall in one bank (atom mod 32
// equal: same atom, or atoms 32 apart) replay that atomic, so terms listed
// around one centre (all angles at an atom, all torsions about a bond)
// serialise.  Greedy: every run of 32 takes, slot by slot, the first
// remaining term whose busiest (role, atom mod 32) count in the run is
// lowest.  Only the order changes; deterministic.
template <class T, class AtomOf>
std::vector<T> spread_terms(const std::vector<T>& v, int roles, AtomOf atom_of) {
  std::vector<T> out;
  out.reserve(v.size());
  std::vector<char> used(v.size(), 0);
  size_t left = v.size();
  while (left > 0) {
    int cnt[4][32] = {};
    for (int slot = 0; slot < 32 && left > 0; ++slot) {
      size_t best = v.size();
      int best_c = 1 << 30;
      for (size_t k = 0; k < v.size() && best_c > 0; ++k) {
        if (used[k]) continue;
        int c = 0;
        for (int r = 0; r < roles; ++r) c = std::max(c, cnt[r][atom_of(v[k], r) & 31]);
        if (c < best_c) {
          best_c = c;
          best = k;
        }
      }
      used[best] = 1;
      --left;
      for (int r = 0; r < roles; ++r) ++cnt[r][atom_of(v[best], r) & 31];
      out.push_back(v[best]);
    }
  }
  return out;
}

// Rotatable bonds of a flexible template (the torsion coordinates of a
// pose).  Root: the lowest-index atom with one bond (atom 0 if none);
// breadth-first search from it, neighbours in increasing index order,
// gives parents and depths.  Candidates: the distinct central bonds of the
// torsion terms in the order of their first term; a candidate is kept when
// it is a search-tree edge (b the parent end, c the child end) that is not
// in a ring, b has a parent and c another neighbour.  Quadruple (parent(b),
// b, c, d), d the lowest-index neighbour of c other than b; moving side:
// atoms reached from c without crossing (b, c).  At most GRIDFF_MAX_ROTORS
// kept, then ordered by the depth of b (stable), so that a rotation only
// moves atoms below every earlier rotor's quadruple.
std::vector<Rotor> template_rotors(int n, const std::vector<std::vector<int>>& adj_in, const int32_t* tors,
                                   int n_tors) {
  std::vector<std::vector<int>> adj = adj_in;
  for (auto& a : adj) std::sort(a.begin(), a.end());
  int root = 0;
  for (int i = 0; i < n; ++i)
    if (adj[i].size() == 1) {
      root = i;
      break;
    }
  std::vector<int> parent(n, -1), depth(n, -1), queue{root};
  depth[root] = 0;
  for (size_t h = 0; h < queue.size(); ++h)
    for (int v : adj[queue[h]])
      if (depth[v] < 0) {
        depth[v] = depth[queue[h]] + 1;
        parent[v] = queue[h];
        queue.push_back(v);
      }
  std::vector<Rotor> kept;
  std::vector<int> kept_depth;
  std::vector<std::pair<int, int>> seen;
  for (int k = 0; k < n_tors && (int)kept.size() < GRIDFF_MAX_ROTORS; ++k) {
    const int j = tors[4 * k + 1], l = tors[4 * k + 2];
    const std::pair<int, int> key(std::min(j, l), std::max(j, l));
    if (std::find(seen.begin(), seen.end(), key) != seen.end()) continue;
    seen.push_back(key);
    int b, c;
    if (parent[l] == j) {
      b = j;
      c = l;
    } else if (parent[j] == l) {
      b = l;
      c = j;
    } else {
      continue;
    }
    if (parent[b] < 0) continue;
    int d = -1;
    for (int v : adj[c])
      if (v != b) {
        d = v;
        break;
      }
    if (d < 0) continue;
    std::vector<char> in(n, 0);
    std::vector<int> stack{c};
    in[c] = 1;
    bool ring = false;
    while (!stack.empty()) {
      const int u = stack.back();
      stack.pop_back();
      for (int v : adj[u]) {
        if (u == c && v == b) continue;
        if (v == b) {
          ring = true;
          continue;
        }
        if (!in[v]) {
          in[v] = 1;
          stack.push_back(v);
        }
      }
    }
    if (ring) continue;
    Rotor R{parent[b], b, c, d, {0u, 0u, 0u, 0u}};
    for (int i = 0; i < n; ++i)
      if (in[i]) R.move[i >> 5] |= 1u << (i & 31);
    kept.push_back(R);
    kept_depth.push_back(depth[b]);
  }
  std::vector<int> order(kept.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return kept_depth[x] < kept_depth[y]; });
  std::vector<Rotor> out;
  for (int i : order) out.push_back(kept[i]);
  return out;
}

// Lab-frame atom positions of rigid replicas: r_i = R(q) b_i + com.
__global__ void rigid_positions_kernel(TemplateView tv, const int* rep_tmpl, const int* rep_off,
                                       const float* pose, int n_rep, float* out) {
  int r = blockIdx.x;
  if (r >= n_rep) return;
  int t = rep_tmpl[r];
  int n = tv.natoms[t], ab = tv.atom_off[t];
  const float* p = pose + 7 * (size_t)r;
  float R[9];
  quat_rot(p[3], p[4], p[5], p[6], R);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float4 b = tv.body[ab + i];
    float* o = out + 3 * ((size_t)rep_off[r] + i);
    o[0] = R[0] * b.x + R[1] * b.y + R[2] * b.z + p[0];
    o[1] = R[3] * b.x + R[4] * b.y + R[5] * b.z + p[1];
    o[2] = R[6] * b.x + R[7] * b.y + R[8] * b.z + p[2];
  }
}

}  // namespace

extern "C" {

gridff_status gridff_replicas_create(gridff_ctx* ctx, int32_t n_templates,
                                     const gridff_molecule* T, int32_t n_rep,
                                     const int32_t* template_of, int32_t rigid, double alpha,
                                     gridff_replicas** out) {
  NvtxRange nvtx_range("gridff_replicas_create");
  if (!ctx || !T || !template_of || !out || n_templates <= 0 || n_rep <= 0)
    return set_err(ctx, GRIDFF_EINVAL, "null argument or empty set");
  *out = nullptr;
  if (!(alpha > 0)) alpha = 1.5;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  // host-side template tables
  std::vector<int> natoms(n_templates), atom_off(n_templates + 1, 0);
  std::vector<float4> body, par, nb, rig(n_templates);
  std::vector<float> rmax(n_templates);
  std::vector<uint32_t> excl;
  std::vector<int> bond_off(1, 0), angle_off(1, 0), tors_off(1, 0);
  std::vector<BondRec> bonds;
  std::vector<AngleRec> angles;
  std::vector<TorsionRec> tors;
  std::vector<int> ub_off(1, 0), ua_off(1, 0), ut_off(1, 0);
  std::vector<BondTerm> ub;
  std::vector<AngleRec> ua;
  std::vector<TorsionRec> ut;
  std::vector<double> tmpl_cost(n_templates);
  std::vector<int> rot_off(1, 0);
  std::vector<Rotor> rot;
  int max_n = 0;
  for (int t = 0; t < n_templates; ++t) {
    const gridff_molecule& m = T[t];
    int n = m.n_atoms;
    if (n < 1 || n > GRIDFF_MAX_ATOMS)
      return set_err(ctx, GRIDFF_EINVAL, "template %d: n_atoms %d outside 1..%d", t, n, GRIDFF_MAX_ATOMS);
    if (!m.xyz || !m.q || !m.R || !m.eps || !m.mass)
      return set_err(ctx, GRIDFF_EINVAL, "template %d: per-atom arrays missing", t);
    max_n = std::max(max_n, n);
    natoms[t] = n;
    atom_off[t + 1] = atom_off[t] + n;
    // adjacency for exclusions (pairs at most two bonds apart)
    std::vector<std::vector<int>> adj(n);
    for (int b = 0; b < m.n_bonds; ++b) {
      int i = m.bonds[2 * b], j = m.bonds[2 * b + 1];
      if (i < 0 || j < 0 || i >= n || j >= n || i == j)
        return set_err(ctx, GRIDFF_EINVAL, "template %d: bond %d has bad atoms", t, b);
      adj[i].push_back(j);
      adj[j].push_back(i);
    }
    std::vector<BondTerm> tub;
    std::vector<AngleRec> tua;
    std::vector<TorsionRec> tut;
    std::vector<std::vector<BondRec>> pb(n);
    std::vector<std::vector<AngleRec>> pa(n);
    std::vector<std::vector<TorsionRec>> pt(n);
    if (!rigid) {
      for (int b = 0; b < m.n_bonds; ++b) {
        int i = m.bonds[2 * b], j = m.bonds[2 * b + 1];
        pb[i].push_back(BondRec{j, 1, m.bond_k[b], m.bond_r0[b]});
        pb[j].push_back(BondRec{i, 0, m.bond_k[b], m.bond_r0[b]});
      }
      for (int a = 0; a < m.n_angles; ++a) {
        const int* A = m.angles + 3 * a;
        for (int k = 0; k < 3; ++k)
          if (A[k] < 0 || A[k] >= n) return set_err(ctx, GRIDFF_EINVAL, "template %d: angle %d", t, a);
        if (A[0] == A[1] || A[1] == A[2] || A[0] == A[2])
          return set_err(ctx, GRIDFF_EINVAL, "template %d: angle %d repeats an atom", t, a);
        for (int role = 0; role < 3; ++role)
          pa[A[role]].push_back(AngleRec{A[0], A[1], A[2], role, m.angle_k[a], m.angle_cos0[a], 0, 0});
        tua.push_back(AngleRec{A[0], A[1], A[2], 0, m.angle_k[a], m.angle_cos0[a], 0, 0});
      }
      for (int b = 0; b < m.n_bonds; ++b)
        tub.push_back(BondTerm{m.bonds[2 * b], m.bonds[2 * b + 1], m.bond_k[b], m.bond_r0[b]});
      for (int a = 0; a < m.n_torsions; ++a) {
        const int* A = m.torsions + 4 * a;
        for (int k = 0; k < 4; ++k)
          if (A[k] < 0 || A[k] >= n) return set_err(ctx, GRIDFF_EINVAL, "template %d: torsion %d", t, a);
        for (int role = 0; role < 4; ++role)
          pt[A[role]].push_back(TorsionRec{A[0], A[1], A[2], A[3], role, m.torsion_n[a],
                                           m.torsion_V[a], m.torsion_cos_nphi0[a]});
        tut.push_back(TorsionRec{A[0], A[1], A[2], A[3], 0, m.torsion_n[a], m.torsion_V[a],
                                m.torsion_cos_nphi0[a]});
      }
    }
    if (!rigid) {
      for (int a = 0; a < m.n_torsions; ++a)
        for (int k = 0; k < 4; ++k)
          if (m.torsions[4 * a + k] < 0 || m.torsions[4 * a + k] >= n)
            return set_err(ctx, GRIDFF_EINVAL, "template %d: torsion %d", t, a);
      const std::vector<Rotor> tr = template_rotors(n, adj, m.torsions, m.n_torsions);
      rot.insert(rot.end(), tr.begin(), tr.end());
    }
    rot_off.push_back((int)rot.size());
    tub = spread_terms(tub, 2, [](const BondTerm& b, int r) { return r == 0 ? b.i : b.j; });
    tua = spread_terms(tua, 3, [](const AngleRec& a, int r) { return r == 0 ? a.a : r == 1 ? a.b : a.c; });
    tut = spread_terms(tut, 4, [](const TorsionRec& q, int r) { return r == 0 ? q.a : r == 1 ? q.b : r == 2 ? q.c : q.d; });
    ub.insert(ub.end(), tub.begin(), tub.end());
    ua.insert(ua.end(), tua.begin(), tua.end());
    ut.insert(ut.end(), tut.begin(), tut.end());
    ub_off.push_back((int)ub.size());
    ua_off.push_back((int)ua.size());
    ut_off.push_back((int)ut.size());
    double M = 0, cx = 0, cy = 0, cz = 0;
    for (int i = 0; i < n; ++i) {
      if (!(m.mass[i] > 0)) return set_err(ctx, GRIDFF_EINVAL, "template %d: mass of atom %d", t, i);
      M += m.mass[i];
      cx += m.mass[i] * m.xyz[3 * i];
      cy += m.mass[i] * m.xyz[3 * i + 1];
      cz += m.mass[i] * m.xyz[3 * i + 2];
    }
    double I[6] = {0, 0, 0, 0, 0, 0};  // xx yy zz xy xz yz
    double rm = 0;
    for (int i = 0; i < n; ++i) {
      double x = m.xyz[3 * i], y = m.xyz[3 * i + 1], z = m.xyz[3 * i + 2], w = m.mass[i];
      I[0] += w * (y * y + z * z);
      I[1] += w * (x * x + z * z);
      I[2] += w * (x * x + y * y);
      I[3] -= w * x * y;
      I[4] -= w * x * z;
      I[5] -= w * y * z;
      rm = std::max(rm, sqrt(x * x + y * y + z * z));
    }
    if (rigid) {
      double tr = I[0] + I[1] + I[2];
      if (fabs(cx) + fabs(cy) + fabs(cz) > 1e-3 * M ||
          fabs(I[3]) + fabs(I[4]) + fabs(I[5]) > 1e-4 * tr + 1e-6)
        return set_err(ctx, GRIDFF_EINVAL,
                       "template %d: rigid body coordinates must be centred at the centre of mass "
                       "and along principal axes", t);
      if (!(I[0] > 0 && I[1] > 0 && I[2] > 0))
        return set_err(ctx, GRIDFF_EINVAL, "template %d: rigid body needs three positive moments", t);
    }
    rig[t] = make_float4((float)M, (float)I[0], (float)I[1], (float)I[2]);
    rmax[t] = (float)std::max(rm, 1e-3);
    // exclusion masks by breadth-first search to depth 2
    for (int i = 0; i < n; ++i) {
      uint32_t w[4] = {0, 0, 0, 0};
      std::vector<int> depth(n, -1);
      std::vector<int> queue{i};
      depth[i] = 0;
      for (size_t h = 0; h < queue.size(); ++h) {
        int u = queue[h];
        if (depth[u] == 2) continue;
        for (int v : adj[u])
          if (depth[v] < 0) {
            depth[v] = depth[u] + 1;
            queue.push_back(v);
          }
      }
      for (int j = 0; j < n; ++j)
        if (depth[j] >= 0) w[j >> 5] |= 1u << (j & 31);
      for (int k = 0; k < 4; ++k) excl.push_back(w[k]);
    }
    // relative cost of one force evaluation (work-queue order): grid quad
    // rounds, nonbonded pair steps, bonded terms per lane
    const double pair_steps = rigid ? 0.0 : (double)((n + 31) / 32) * (n / 2);
    tmpl_cost[t] = 3.0 * ((n + 7) / 8) + pair_steps + 2.0 * (ub_off[t + 1] - ub_off[t]) / 32.0 +
                   3.0 * (ua_off[t + 1] - ua_off[t]) / 32.0 + 6.0 * (ut_off[t + 1] - ut_off[t]) / 32.0;
    for (int i = 0; i < n; ++i) {
      double R = m.R[i], eps = m.eps[i];
      body.push_back(make_float4(m.xyz[3 * i], m.xyz[3 * i + 1], m.xyz[3 * i + 2], m.mass[i]));
      // Eq. V_Morse: P_i = eps_i e^{2 alpha R_i}, L_i = -2 eps_i e^{alpha R_i}
      par.push_back(make_float4(m.q[i], (float)(eps * exp(2 * alpha * R)),
                                (float)(-2 * eps * exp(alpha * R)), 0.f));
      nb.push_back(make_float4(m.q[i], m.R[i], m.eps[i], 0.f));
      for (auto& b : pb[i]) bonds.push_back(b);
      for (auto& a : pa[i]) angles.push_back(a);
      for (auto& a : pt[i]) tors.push_back(a);
      bond_off.push_back((int)bonds.size());
      angle_off.push_back((int)angles.size());
      tors_off.push_back((int)tors.size());
    }
  }
  std::vector<int> rep_tmpl(n_rep), rep_off(n_rep + 1, 0);
  for (int r = 0; r < n_rep; ++r) {
    int t = template_of[r];
    if (t < 0 || t >= n_templates) return set_err(ctx, GRIDFF_EINVAL, "replica %d: template %d", r, t);
    rep_tmpl[r] = t;
    rep_off[r + 1] = rep_off[r] + natoms[t];
  }
  std::vector<int> order(n_rep);
  for (int r = 0; r < n_rep; ++r) order[r] = r;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return tmpl_cost[rep_tmpl[a]] > tmpl_cost[rep_tmpl[b]]; });
  // one device blob for the templates
  std::vector<unsigned char> blob;
  size_t o_nat = push(blob, natoms), o_aoff = push(blob, atom_off), o_body = push(blob, body),
         o_par = push(blob, par), o_nb = push(blob, nb), o_ex = push(blob, excl),
         o_boff = push(blob, bond_off), o_b = push(blob, bonds), o_aof = push(blob, angle_off),
         o_a = push(blob, angles), o_tof = push(blob, tors_off), o_t = push(blob, tors),
         o_rig = push(blob, rig), o_rmax = push(blob, rmax), o_ubo = push(blob, ub_off), o_ub = push(blob, ub), o_uao = push(blob, ua_off),
         o_ua = push(blob, ua), o_uto = push(blob, ut_off), o_ut = push(blob, ut), o_ord = push(blob, order),
         o_roff = push(blob, rot_off), o_rot = push(blob, rot);
  gridff_replicas* R = new gridff_replicas();
  R->ctx = ctx;
  R->device = ctx->device;
  R->n_rep = n_rep;
  R->n_atoms = rep_off[n_rep];
  R->n_tmpl = n_templates;
  R->rigid = rigid ? 1 : 0;
  R->alpha = (float)alpha;
  R->max_natoms = max_n;
  auto bail = [&](gridff_status st, const char* what) {
    gridff_replicas_destroy(R);
    return set_err(ctx, st, "%s", what);
  };
  if (cudaMalloc(&R->tmpl_blob, blob.size()) != cudaSuccess) return bail(GRIDFF_ENOMEM, "templates");
  if (cudaMemcpyAsync(R->tmpl_blob, blob.data(), blob.size(), cudaMemcpyHostToDevice, ctx->stream))
    return bail(GRIDFF_ECUDA, "template upload");
  unsigned char* B = (unsigned char*)R->tmpl_blob;
  R->tv.natoms = (const int*)(B + o_nat);
  R->tv.atom_off = (const int*)(B + o_aoff);
  R->tv.body = (const float4*)(B + o_body);
  R->tv.par = (const float4*)(B + o_par);
  R->tv.nb = (const float4*)(B + o_nb);
  R->tv.excl = (const uint32_t*)(B + o_ex);
  R->tv.bond_off = (const int*)(B + o_boff);
  R->tv.bonds = (const BondRec*)(B + o_b);
  R->tv.angle_off = (const int*)(B + o_aof);
  R->tv.angles = (const AngleRec*)(B + o_a);
  R->tv.tors_off = (const int*)(B + o_tof);
  R->tv.tors = (const TorsionRec*)(B + o_t);
  R->tv.rigid = (const float4*)(B + o_rig);
  R->tv.rmax = (const float*)(B + o_rmax);
  R->tv.ub_off = (const int*)(B + o_ubo);
  R->tv.ub = (const BondTerm*)(B + o_ub);
  R->tv.ua_off = (const int*)(B + o_uao);
  R->tv.ua = (const AngleRec*)(B + o_ua);
  R->tv.ut_off = (const int*)(B + o_uto);
  R->tv.ut = (const TorsionRec*)(B + o_ut);
  R->order = (int*)(B + o_ord);
  R->tv.rot_off = (const int*)(B + o_roff);
  R->tv.rot = (const Rotor*)(B + o_rot);
  R->h_rot_off = new int[n_templates + 1];
  memcpy(R->h_rot_off, rot_off.data(), (n_templates + 1) * sizeof(int));
  R->h_rot = new Rotor[rot.size() + 1];
  if (!rot.empty()) memcpy(R->h_rot, rot.data(), rot.size() * sizeof(Rotor));
  R->tv.alpha = (float)alpha;
  size_t nx = rigid ? 7 * (size_t)n_rep : 3 * (size_t)R->n_atoms;
  size_t nv = rigid ? 6 * (size_t)n_rep : 3 * (size_t)R->n_atoms;
  if (cudaMalloc(&R->rep_tmpl, n_rep * sizeof(int)) || cudaMalloc(&R->rep_off, (n_rep + 1) * sizeof(int)) ||
      cudaMalloc(&R->x, nx * sizeof(float)) || cudaMalloc(&R->v, nv * sizeof(float)) ||
      cudaMalloc(&R->fire_dt, n_rep * sizeof(float)) || cudaMalloc(&R->fire_alpha, n_rep * sizeof(float)) ||
      cudaMalloc(&R->fire_nplus, n_rep * sizeof(int)) || cudaMalloc(&R->status, n_rep * sizeof(int)) ||
      cudaMalloc(&R->steps, n_rep * sizeof(int)) || cudaMalloc(&R->energy, n_rep * sizeof(double)) ||
      cudaMalloc(&R->handoff, n_rep * sizeof(int)) || cudaMalloc(&R->handoff_p, n_rep * sizeof(float4)) ||
      cudaMalloc(&R->last_x, nx * sizeof(float)) || cudaMalloc(&R->last_f, nv * sizeof(float)))
    return bail(GRIDFF_ENOMEM, "replica state");
  R->h_rep_off = new int[n_rep + 1];
  memcpy(R->h_rep_off, rep_off.data(), (n_rep + 1) * sizeof(int));
  cudaStream_t s = ctx->stream;
  if (cudaMemcpyAsync(R->rep_tmpl, rep_tmpl.data(), n_rep * sizeof(int), cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(R->rep_off, rep_off.data(), (n_rep + 1) * sizeof(int), cudaMemcpyHostToDevice, s) ||
      cudaMemsetAsync(R->x, 0, nx * sizeof(float), s) || cudaMemsetAsync(R->v, 0, nv * sizeof(float), s) ||
      cudaMemsetAsync(R->fire_dt, 0, n_rep * sizeof(float), s) ||
      cudaMemsetAsync(R->fire_alpha, 0, n_rep * sizeof(float), s) ||
      cudaMemsetAsync(R->fire_nplus, 0, n_rep * sizeof(int), s) ||
      cudaMemsetAsync(R->status, 0, n_rep * sizeof(int), s) ||
      cudaMemsetAsync(R->steps, 0, n_rep * sizeof(int), s) ||
      cudaMemsetAsync(R->energy, 0, n_rep * sizeof(double), s) ||
      cudaMemsetAsync(R->last_x, 0xff, nx * sizeof(float), s) ||   // all bits set: NaN (nothing recorded)
      cudaMemsetAsync(R->last_f, 0xff, nv * sizeof(float), s))
    return bail(GRIDFF_ECUDA, "replica init");
  if (rigid) {
    // identity orientation
    std::vector<float> pose(nx, 0.f);
    for (int r = 0; r < n_rep; ++r) pose[7 * r + 3] = 1.f;
    if (cudaMemcpyAsync(R->x, pose.data(), nx * sizeof(float), cudaMemcpyHostToDevice, s))
      return bail(GRIDFF_ECUDA, "pose init");
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return bail(GRIDFF_ECUDA, "replica init sync");
  *out = R;
  return GRIDFF_OK;
}

gridff_status gridff_template_factors(const gridff_replicas* R, int32_t t, float* qpl) {
  if (!R || !qpl || t < 0 || t >= R->n_tmpl) return GRIDFF_EINVAL;
  gridff_ctx* ctx = R->ctx;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  int off[2];
  GRIDFF_CUDA(ctx, cudaMemcpy(off, R->tv.atom_off + t, 2 * sizeof(int), cudaMemcpyDeviceToHost));
  std::vector<float4> par(off[1] - off[0]);
  if (!par.empty())
    GRIDFF_CUDA(ctx, cudaMemcpy(par.data(), R->tv.par + off[0], par.size() * sizeof(float4), cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < par.size(); ++i) {
    qpl[3 * i] = par[i].x;
    qpl[3 * i + 1] = par[i].y;
    qpl[3 * i + 2] = par[i].z;
  }
  return GRIDFF_OK;
}

void gridff_replicas_destroy(gridff_replicas* R) {
  if (!R) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(R->device);
  void* ptrs[] = {R->tmpl_blob, R->rep_tmpl, R->rep_off, R->x, R->v, R->fire_dt, R->fire_alpha,
                  R->fire_nplus, R->status, R->steps, R->energy, R->handoff, R->handoff_p,
                  R->last_x, R->last_f, R->gval, R->gkey};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  cudaSetDevice(prev);
  cudaGetLastError();   // leave no error of this teardown behind
  delete[] R->h_rep_off;
  delete[] R->h_rot_off;
  delete[] R->h_rot;
  delete R;
}

gridff_status gridff_replicas_info(const gridff_replicas* R, int32_t* n_rep, int32_t* n_atoms,
                                   int32_t* atom_offset) {
  if (!R) return GRIDFF_EINVAL;
  if (n_rep) *n_rep = R->n_rep;
  if (n_atoms) *n_atoms = R->n_atoms;
  if (atom_offset) memcpy(atom_offset, R->h_rep_off, (R->n_rep + 1) * sizeof(int));
  return GRIDFF_OK;
}

gridff_status gridff_set_state(gridff_replicas* R, const float* x, const float* v, int flags) {
  if (!R || !x) return set_err(R ? R->ctx : nullptr, GRIDFF_EINVAL, "null argument");
  gridff_ctx* ctx = R->ctx;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  size_t nx = R->rigid ? 7 * (size_t)R->n_rep : 3 * (size_t)R->n_atoms;
  size_t nv = R->rigid ? 6 * (size_t)R->n_rep : 3 * (size_t)R->n_atoms;
  if (!copy_in(ctx, R->x, x, nx * sizeof(float), flags)) return set_err(ctx, GRIDFF_ECUDA, "state copy");
  if (v) {
    if (!copy_in(ctx, R->v, v, nv * sizeof(float), flags)) return set_err(ctx, GRIDFF_ECUDA, "state copy");
  } else {
    GRIDFF_CUDA(ctx, cudaMemsetAsync(R->v, 0, nv * sizeof(float), ctx->stream));
  }
  return finish(ctx, flags);
}

gridff_status gridff_get_state(gridff_replicas* R, float* x, float* v, int flags) {
  if (!R || !x) return set_err(R ? R->ctx : nullptr, GRIDFF_EINVAL, "null argument");
  gridff_ctx* ctx = R->ctx;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  size_t nx = R->rigid ? 7 * (size_t)R->n_rep : 3 * (size_t)R->n_atoms;
  size_t nv = R->rigid ? 6 * (size_t)R->n_rep : 3 * (size_t)R->n_atoms;
  if (!copy_out(ctx, x, R->x, nx * sizeof(float), flags)) return set_err(ctx, GRIDFF_ECUDA, "state copy");
  if (v && !copy_out(ctx, v, R->v, nv * sizeof(float), flags))
    return set_err(ctx, GRIDFF_ECUDA, "state copy");
  return finish(ctx, flags);
}

gridff_status gridff_get_positions(gridff_replicas* R, float* x, int flags) {
  if (!R || !x) return set_err(R ? R->ctx : nullptr, GRIDFF_EINVAL, "null argument");
  gridff_ctx* ctx = R->ctx;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  size_t bytes = 3 * (size_t)R->n_atoms * sizeof(float);
  if (!R->rigid) {
    if (!copy_out(ctx, x, R->x, bytes, flags)) return set_err(ctx, GRIDFF_ECUDA, "copy");
    return finish(ctx, flags);
  }
  float* dst = x;
  float* tmp = nullptr;
  if (!(flags & GRIDFF_DEVICE_PTRS)) {
    GRIDFF_CUDA(ctx, cudaMallocAsync(&tmp, bytes, ctx->stream));
    dst = tmp;
  }
  rigid_positions_kernel<<<R->n_rep, 64, 0, ctx->stream>>>(R->tv, R->rep_tmpl, R->rep_off, R->x,
                                                           R->n_rep, dst);
  cudaError_t e = cudaGetLastError();
  if (tmp) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(x, tmp, bytes, cudaMemcpyDeviceToHost, ctx->stream);
    const cudaError_t ef = cudaFreeAsync(tmp, ctx->stream);
    if (e == cudaSuccess) e = ef;
  }
  if (e != cudaSuccess) return set_err(ctx, GRIDFF_ECUDA, "positions: %s", cudaGetErrorString(e));
  return finish(ctx, flags);
}

gridff_status gridff_get_last_eval(gridff_replicas* R, float* x, float* f, int flags) {
  if (!R) return GRIDFF_EINVAL;
  gridff_ctx* ctx = R->ctx;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  size_t nx = R->rigid ? 7 * (size_t)R->n_rep : 3 * (size_t)R->n_atoms;
  size_t nf = R->rigid ? 6 * (size_t)R->n_rep : 3 * (size_t)R->n_atoms;
  bool ok = true;
  if (x) ok &= copy_out(ctx, x, R->last_x, nx * sizeof(float), flags);
  if (f) ok &= copy_out(ctx, f, R->last_f, nf * sizeof(float), flags);
  if (!ok) return set_err(ctx, GRIDFF_ECUDA, "copy");
  return finish(ctx, flags);
}

gridff_status gridff_get_fire_state(gridff_replicas* R, float* dt, float* alpha, int32_t* nplus,
                                    int32_t* status, int32_t* steps, double* energy, int flags) {
  if (!R) return GRIDFF_EINVAL;
  gridff_ctx* ctx = R->ctx;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  size_t n = R->n_rep;
  bool ok = true;
  if (dt) ok &= copy_out(ctx, dt, R->fire_dt, n * sizeof(float), flags);
  if (alpha) ok &= copy_out(ctx, alpha, R->fire_alpha, n * sizeof(float), flags);
  if (nplus) ok &= copy_out(ctx, nplus, R->fire_nplus, n * sizeof(int), flags);
  if (status) ok &= copy_out(ctx, status, R->status, n * sizeof(int), flags);
  if (steps) ok &= copy_out(ctx, steps, R->steps, n * sizeof(int), flags);
  if (energy) ok &= copy_out(ctx, energy, R->energy, n * sizeof(double), flags);
  if (!ok) return set_err(ctx, GRIDFF_ECUDA, "copy");
  return finish(ctx, flags);
}

}  // extern "C"
