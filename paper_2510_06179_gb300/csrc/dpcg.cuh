// a2 (blocks), a3 and a4 distributed over a thread-block cluster: Algorithm 4 for one OCP whose
// workspace does not fit in one CTA's shared memory (12-state rigid body, T up to a few hundred).
// CTA 0 of the cluster (the leader) runs every other stage of the SQP iteration and the backward
// pass from the OCP's global-memory workspace, as the single-team kernel does.  At each PCG solve
// it hands the solve to all CTAs of the cluster: CTA r copies the factors A_t, B_t and the FP64
// vectors of the knots [r KC, (r+1) KC) into its own shared memory, forms their Schur and
// preconditioner blocks there (or reads stored ones), and the PCG then runs with every block
// resident on chip:
//   - knot k's row of S p (and of Phi^-1 r) needs p_{k-1} and the product with block k+1; a CTA
//     keeps the first block of the next CTA as a halo copy, and the owner of a boundary knot
//     sends the vector values its neighbours need into their shared memory along with the next
//     all-reduce, so the halos cost no extra synchronisation;
//   - each of the two dot products of an iteration is an all-reduce: warp shuffles, one partial
//     per warp, then every CTA stores its partial into a slot of every CTA with an asynchronous
//     DSMEM store that completes bytes on the receiver's mbarrier (st.async), so a phase is done
//     when all bytes it expects (partials and halo values) have landed; every CTA sums the slots
//     in rank order, so all CTAs hold bitwise the same totals and take the same decisions;
//   - the updates p = z + beta p and r = r - alpha y are applied where they are consumed (each
//     thread forms the values of the three knots its block row reads, from double-buffered
//     vectors), so an iteration synchronises only at its two all-reduces;
//   - reliable updates evaluate the FP64 true residual gamma - H G^-1 H^T lambda from the
//     factors (hp_apply's two passes, distributed the same way); when the stagnation test fires,
//     the double-float PCG (stage_pcg_df's iteration) continues on the cluster the same way.
// Every wait on another CTA is an mbarrier wait with a time limit; when one runs out the CTA
// stops waiting from then on, and the OCP is flagged (ST_SYNC_TIMEOUT).
#pragma once
#include "cluster.cuh"

namespace dmpc {

constexpr int kClMaxCtas = 8;     // CTAs per cluster (the portable cluster size)
constexpr int kClThreads = 256;   // threads per CTA (the leader's team)
constexpr int kClRows = 2;        // rows of a knot's block row per thread
constexpr int kClNV = 3;          // widest all-reduce
constexpr unsigned long long kClWaitNs = 4000000000ull;  // time limit of one wait (4 s)
constexpr int ST_SYNC_TIMEOUT = 256;

#ifdef DMPC_CLUSTER_PCG
constexpr bool kClusterPcg = true;
#else
constexpr bool kClusterPcg = false;
#endif

enum ClCommand : int { CL_PCG = 1, CL_EXIT = 2 };
// mbarriers of a CTA: two for the all-reduce phases (alternating), the leader's command, and a
// release barrier for the end of a solve (global-memory write-back)
enum ClBar : int { CB_RED0 = 0, CB_RED1 = 1, CB_CMD = 2, CB_REL = 3 };

// Shared-memory layout of one CTA of the cluster (float offsets unless noted).  KC = knot
// capacity per CTA.  Blocks are knot-minor over KB = KC + 1 slots (slot nk holds the next CTA's
// first knot); vectors over KV = KC + 2 slots (slot 0 and nk + 1 are halo slots, own knots at
// 1..nk).  P and R are double-buffered.
struct ClLayout {
  int KC, KB, KV;
  int D, O, Pd, Po, A, Bm;   // float blocks
  int Pv[2], R[2], Y, Z, DL; // float vectors
  int rh, yh, zh, ph;        // halo staging, [side][NX]: side 0 = previous CTA, 1 = next CTA
  int Lf, Wf;                // per-knot scratch of the block inversion (Cholesky factor, its inverse)
  // double-float rescue (aliases the inversion scratch): vectors X, R, P, Y, Z, WX, WU (one hi/lo
  // float pair per element, element i of vector slot j at 2 (i KV + j)) and halo staging
  // [side][NX] pairs for r, y, z, p
  int dX, dR, dP, dY, dZ, dWX, dWU, drh, dyh, dzh, dph;
  int pdp;                   // the previous CTA's last Phi^-1 diagonal block (NX x NX)
  int misc;                  // copy of the OCP's scalars (weights, reciprocals)
  int wpart, slots;          // all-reduce scratch: 2 x warps x kClNV, 2 x kClMaxCtas x kClNV
  int job;                   // command words written by the leader
  int bars;                  // four mbarriers (ClBar)
  int dbase;                 // float offset of the double region
  int LP, G, WX, WU;         // double vectors (offsets in doubles from dbase)
  int total;
};

__host__ __device__ inline ClLayout cl_layout(int nx, int nu, int kc) {
  ClLayout S;
  S.KC = kc;
  S.KB = kc + 1;
  S.KV = kc + 2;
  int f = 0;
  const int b = nx * nx * S.KB;
  S.D = f; f += b;
  S.O = f; f += b;
  S.Pd = f; f += b;
  S.Po = f; f += b;
  S.A = f; f += b;
  S.Bm = f; f += nx * nu * S.KB;
  const int v = nx * S.KV;
  S.Pv[0] = f; f += v;
  S.Pv[1] = f; f += v;
  S.R[0] = f; f += v;
  S.R[1] = f; f += v;
  S.Y = f; f += v;
  S.Z = f; f += v;
  S.DL = f; f += v;
  S.rh = f; f += 2 * nx;
  S.yh = f; f += 2 * nx;
  S.zh = f; f += 2 * nx;
  S.ph = f; f += 2 * nx;
  S.Lf = f;
  S.Wf = f + nx * nx * S.KB;
  {
    int g = f;
    const int dv = 2 * nx * S.KV;
    S.dX = g; g += dv;
    S.dR = g; g += dv;
    S.dP = g; g += dv;
    S.dY = g; g += dv;
    S.dZ = g; g += dv;
    S.dWX = g; g += dv;
    S.dWU = g; g += 2 * nu * S.KV;
    S.drh = g; g += 4 * nx;
    S.dyh = g; g += 4 * nx;
    S.dzh = g; g += 4 * nx;
    S.dph = g; g += 4 * nx;
    f = (g > f + 2 * nx * nx * S.KB) ? g : f + 2 * nx * nx * S.KB;
  }
  S.pdp = f; f += nx * nx;
  f = (f + 3) & ~3;
  S.misc = f; f += kMisc;
  S.wpart = f; f += 2 * (kClThreads / 32) * kClNV;
  S.slots = f; f += 2 * kClMaxCtas * kClNV;
  S.job = f; f += 8;
  f = (f + 3) & ~3;
  S.bars = f; f += 8;
  S.dbase = f;
  int d = 0;
  S.LP = d; d += nx * S.KV;
  S.G = d; d += nx * S.KV;
  S.WX = d; d += nx * S.KV;
  S.WU = d; d += nu * S.KV;
  f += 2 * d;
  S.total = (f + 3) & ~3;
  return S;
}

// Largest knot count per CTA: one thread per (knot, group of kClRows rows).
__host__ __device__ constexpr int cl_max_kc(int nx) { return kClThreads / (nx / kClRows); }

// Per-thread state of the distributed PCG in one CTA.
template <class M>
struct ClRun {
  static constexpr int NX = M::NX, NU = M::NU, RG = NX / kClRows;
  float* sm;
  double* dm;
  ClLayout S;
  uint32_t rank, ncta;
  int tid;
  int phase;        // all-reduce phase counter
  uint32_t cmd_par; // parity of the next command phase (followers)
  uint32_t rel_par; // parity of the next release-barrier phase
  bool broken;      // a wait ran out: no more waiting in this CTA
  // current OCP
  int K, T, KC, k0, nk, kl, r0;
  bool act, has_prev, has_next;

  __device__ __forceinline__ float* F(int off) const { return sm + off; }
  __device__ __forceinline__ double* Dd(int off) const { return dm + off; }
  __device__ __forceinline__ uint32_t bar(int i) const { return cl::saddr(sm + S.bars) + 8u * (uint32_t)i; }
  __device__ __forceinline__ double qinv(int k, int i) const {
    return reinterpret_cast<const double*>(sm + S.misc + MS_DINV)[(k < T ? 0 : 24) + i];
  }
  __device__ __forceinline__ double rinv(int i) const {
    return reinterpret_cast<const double*>(sm + S.misc + MS_DINV)[16 + i];
  }
  // shared::cluster address of float `off` (or double `doff`) of CTA `q`'s shared memory
  __device__ __forceinline__ uint32_t remote(int off, uint32_t q) const { return cl::map(cl::saddr(sm + off), q); }
  __device__ __forceinline__ uint32_t remote_d(int doff, uint32_t q) const { return cl::map(cl::saddr(dm + doff), q); }
  // the all-reduce mbarrier of the coming phase in CTA q
  __device__ __forceinline__ uint32_t red_bar(uint32_t q) const { return cl::map(bar(phase & 1), q); }

  __device__ void init(float* smem, int kc) {
    sm = smem;
    S = cl_layout(NX, NU, kc);
    dm = reinterpret_cast<double*>(smem + S.dbase);
    rank = cl::rank();
    ncta = cl::ncta();
    tid = threadIdx.x;
    phase = 0;
    cmd_par = 0;
    rel_par = 0;
    broken = false;
  }
  // knot partition of an OCP with K knots over the cluster's CTAs
  __device__ void bind(int K_, int T_) {
    K = K_;
    T = T_;
    KC = (K + (int)ncta - 1) / (int)ncta;
    k0 = (int)rank * KC;
    nk = K - k0;
    nk = nk < 0 ? 0 : (nk > KC ? KC : nk);
    act = nk > 0 && tid < RG * nk;
    kl = act ? tid % nk : 0;
    r0 = act ? (tid / nk) * kClRows : 0;
    has_prev = nk > 0 && k0 > 0;
    has_next = nk > 0 && k0 + nk < K;
  }
  // bytes of halo values this CTA receives in a phase where each existing neighbour sends
  // `per_side` bytes
  __device__ __forceinline__ uint32_t halo_bytes(uint32_t per_side) const {
    return per_side * ((has_prev ? 1u : 0u) + (has_next ? 1u : 0u));
  }
};

// Sum NV values over every thread of every CTA of the cluster; all threads of all CTAs receive
// bitwise the same totals.  halo_rx: bytes of halo values other CTAs send to this one in the same
// phase (their st.async stores signal the same mbarrier), which are visible after the call.
template <class M, int NV>
__device__ __forceinline__ void cl_sum(ClRun<M>& r, float (&v)[NV], uint32_t halo_rx) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], off);
  }
  const int b = r.phase & 1;
  const uint32_t par = (uint32_t)(r.phase >> 1) & 1u;
  float* wp = r.F(r.S.wpart) + b * (kClThreads / 32) * kClNV;
  float* sl = r.F(r.S.slots) + b * kClMaxCtas * kClNV;
  if ((r.tid & 31) == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) wp[(r.tid >> 5) * kClNV + j] = v[j];
  }
  __syncthreads();
  if (r.tid < (int)r.ncta && !r.broken) {
    float s[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) s[j] = 0.f;
    for (int q = 0; q < kClThreads / 32; ++q) {
#pragma unroll
      for (int j = 0; j < NV; ++j) s[j] += wp[q * kClNV + j];
    }
    const uint32_t dst = r.remote(r.S.slots + b * kClMaxCtas * kClNV + (int)r.rank * kClNV, (uint32_t)r.tid);
    const uint32_t rb = r.red_bar((uint32_t)r.tid);
#pragma unroll
    for (int j = 0; j < NV; ++j) cl::st_async_f32(dst + 4u * (uint32_t)j, s[j], rb);
  }
  if (r.tid == 0 && !r.broken) cl::arrive_expect_tx(r.bar(b), r.ncta * NV * 4u + halo_rx);
  bool ok = r.broken ? false : cl::wait(r.bar(b), par, kClWaitNs);
  ok = __syncthreads_and(ok) != 0;
  if (!ok) r.broken = true;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    float t = 0.f;
    for (uint32_t q = 0; q < r.ncta; ++q) t += sl[q * kClNV + j];
    v[j] = t;
  }
  ++r.phase;
}

template <class M>
__device__ __forceinline__ void cl_barrier(ClRun<M>& r, uint32_t halo_rx) {
  float d[1] = {0.f};
  cl_sum<M, 1>(r, d, halo_rx);
}

// Release barrier over the cluster: every thread's earlier writes (global memory included) are
// visible to every thread of the cluster after it.
template <class M>
__device__ __forceinline__ void cl_release_barrier(ClRun<M>& r) {
  __syncthreads();
  if (r.tid < (int)r.ncta && !r.broken) cl::arrive_remote(cl::map(r.bar(CB_REL), (uint32_t)r.tid));
  bool ok = true;
  if (r.tid == 0) ok = r.broken ? false : cl::wait(r.bar(CB_REL), r.rel_par, kClWaitNs);
  ok = __syncthreads_and(ok) != 0;
  if (!ok) r.broken = true;
  r.rel_par ^= 1u;
}

// Send this thread's rows of a boundary knot's values (a, b) into the staging arrays of the
// neighbouring CTAs (side 1 of the previous CTA, side 0 of the next CTA) for the coming phase.
template <class M>
__device__ __forceinline__ void cl_push_pair(ClRun<M>& r, int st_a, int st_b, const float* a, const float* b) {
  constexpr int NX = M::NX;
  if (!r.act || r.broken) return;
  if (r.kl == 0 && r.has_prev) {
    const uint32_t q = r.rank - 1, rb = r.red_bar(q);
    const uint32_t da = r.remote(st_a + NX + r.r0, q), db = r.remote(st_b + NX + r.r0, q);
#pragma unroll
    for (int i = 0; i < kClRows; ++i) { cl::st_async_f32(da + 4u * i, a[i], rb); cl::st_async_f32(db + 4u * i, b[i], rb); }
  }
  if (r.kl == r.nk - 1 && r.has_next) {
    const uint32_t q = r.rank + 1, rb = r.red_bar(q);
    const uint32_t da = r.remote(st_a + r.r0, q), db = r.remote(st_b + r.r0, q);
#pragma unroll
    for (int i = 0; i < kClRows; ++i) { cl::st_async_f32(da + 4u * i, a[i], rb); cl::st_async_f32(db + 4u * i, b[i], rb); }
  }
}

// Rows [r0, r0 + kClRows) of the symmetric block-tridiagonal row of knot kl:
// out = Md_k v_k + Mo_k v_{k-1} + Mo_{k+1}^T v_{k+1} (block slots kl and kl + 1; missing
// neighbours are zero blocks and zero vectors).
template <class M>
__device__ __forceinline__ void cl_block_rows(const ClRun<M>& r, int md, int mo, const float (&vm)[M::NX],
                                              const float (&vc)[M::NX], const float (&vp)[M::NX],
                                              float (&out)[kClRows]) {
  constexpr int NX = M::NX;
  const int KB = r.S.KB, kl = r.kl;
  const float* Md = r.F(md);
  const float* Mo = r.F(mo);
#pragma unroll
  for (int q = 0; q < kClRows; ++q) {
    const int i = r.r0 + q;
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < NX; ++j) acc = fmaf(Md[(i * NX + j) * KB + kl], vc[j], acc);
#pragma unroll
    for (int j = 0; j < NX; ++j) acc = fmaf(Mo[(i * NX + j) * KB + kl], vm[j], acc);
#pragma unroll
    for (int j = 0; j < NX; ++j) acc = fmaf(Mo[(j * NX + i) * KB + kl + 1], vp[j], acc);
    out[q] = acc;
  }
}

// Values x = a + s b of knots kl - 1, kl, kl + 1 (vector arrays a, b over the vector slots; a
// halo knot from the staging arrays ha, hb of its side, which stay zero when the side has no
// neighbour).  The source of each knot is chosen by pointer, so every value costs two loads.
template <class M>
__device__ __forceinline__ void cl_gather(const ClRun<M>& r, const float* a, const float* b, float s, const float* ha,
                                          const float* hb, float (&xm)[M::NX], float (&xc)[M::NX],
                                          float (&xp)[M::NX]) {
  constexpr int NX = M::NX;
  const int KV = r.S.KV, sl = r.kl + 1;
  const bool first = r.kl == 0, last = r.kl == r.nk - 1;
  const float* am = first ? ha : a + sl - 1;
  const float* bm = first ? hb : b + sl - 1;
  const float* ap = last ? ha + NX : a + sl + 1;
  const float* bp = last ? hb + NX : b + sl + 1;
  const int sm_ = first ? 1 : KV, sp_ = last ? 1 : KV;
#pragma unroll
  for (int j = 0; j < NX; ++j) {
    xc[j] = fmaf(s, b[j * KV + sl], a[j * KV + sl]);
    xm[j] = fmaf(s, bm[j * sm_], am[j * sm_]);
    xp[j] = fmaf(s, bp[j * sp_], ap[j * sp_]);
  }
}

// First half of an iteration: p = z + beta p_old (formed where read), own rows of p into
// Pv[pnew], y = S p rows into Y; returns this thread's share of p^T y and sends the boundary
// knots' r (current, R[rcur]) and y to the neighbours.
template <class M>
__device__ __forceinline__ float cl_step_sp(ClRun<M>& r, int pold, int pnew, int rcur, float beta) {
  constexpr int NX = M::NX;
  if (!r.act) return 0.f;
  const int KV = r.S.KV, sl = r.kl + 1;
  float pm[NX], pc[NX], pp[NX], y[kClRows], rv[kClRows];
  cl_gather<M>(r, r.F(r.S.Z), r.F(r.S.Pv[pold]), beta, r.F(r.S.zh), r.F(r.S.ph), pm, pc, pp);
  cl_block_rows<M>(r, r.S.D, r.S.O, pm, pc, pp, y);
  float v = 0.f;
#pragma unroll
  for (int q = 0; q < kClRows; ++q) {
    const int i = r.r0 + q;
    r.F(r.S.Pv[pnew])[i * KV + sl] = pc[i];
    r.F(r.S.Y)[i * KV + sl] = y[q];
    v = fmaf(pc[i], y[q], v);
    rv[q] = r.F(r.S.R[rcur])[i * KV + sl];
  }
  cl_push_pair<M>(r, r.S.rh, r.S.yh, rv, y);
  return v;
}

// Second half: r_new = r - alpha y (formed where read; own rows into R[rnew] and dl += alpha p
// when UPD), z = Phi^-1 r_new rows into Z; returns the share of r_new^T z and sends the boundary
// knots' z and p (Pv[pcur]) to the neighbours.  Without UPD r is R[rcur] as it stands (after a
// true-residual replacement; halos from the staging with y = 0).
template <class M, bool UPD>
__device__ __forceinline__ float cl_step_pc(ClRun<M>& r, int rcur, int rnew, int pcur, float alpha) {
  constexpr int NX = M::NX;
  if (!r.act) return 0.f;
  const int KV = r.S.KV, sl = r.kl + 1;
  float rm[NX], rc[NX], rp[NX], z[kClRows], pv[kClRows];
  const float* Rc = r.F(r.S.R[rcur]);
  if (UPD) cl_gather<M>(r, Rc, r.F(r.S.Y), -alpha, r.F(r.S.rh), r.F(r.S.yh), rm, rc, rp);
  else cl_gather<M>(r, Rc, Rc, 0.f, r.F(r.S.rh), r.F(r.S.rh), rm, rc, rp);
  cl_block_rows<M>(r, r.S.Pd, r.S.Po, rm, rc, rp, z);
  float e = 0.f;
#pragma unroll
  for (int q = 0; q < kClRows; ++q) {
    const int i = r.r0 + q;
    pv[q] = r.F(r.S.Pv[pcur])[i * KV + sl];
    if (UPD) {
      r.F(r.S.R[rnew])[i * KV + sl] = rc[i];
      r.F(r.S.DL)[i * KV + sl] = fmaf(alpha, pv[q], r.F(r.S.DL)[i * KV + sl]);
    }
    r.F(r.S.Z)[i * KV + sl] = z[q];
    e = fmaf(rc[i], z[q], e);
  }
  cl_push_pair<M>(r, r.S.zh, r.S.ph, z, pv);
  return e;
}

// FP64 true residual R[rb] = gamma - H G^-1 H^T LP on the own knots (hp_apply's two passes),
// leaving WX, WU = H^T LP; halos: the next CTA's first LP (sent when push_lp, else already in
// place), the previous CTA's last WX, WU, and both neighbours' new R (sent into the staging with
// y = 0).  Three phases (two without push_lp).
// a2 and a3 on the cluster: each CTA forms the Schur blocks D_k, O_k (Eq. 10, FP32, from the
// factors A_t, B_t and the projected weights) of its own knots and of the next CTA's first knot
// (O only), then Phi^-1: Pd_k = D_k^-1 by a Cholesky factorisation whose rows are shared by the
// knot's threads (column by column), and Po_k = -D_k^-1 O_k D_{k-1}^-1 with the previous CTA's
// last D^-1 read over DSMEM.  Element by element the arithmetic is that of stage_schur,
// stage_precond and spd_inverse.  Returns whether a diagonal block of this CTA failed Cholesky
// (its inverse is then the inverse of its diagonal, as in spd_inverse).
template <class M>
__device__ __noinline__ bool cl_form_blocks(ClRun<M>& r) {
  constexpr int NX = M::NX, NU = M::NU;
  const int KB = r.S.KB, kl = r.kl, k = r.k0 + kl, nk = r.nk;
  float* D = r.F(r.S.D);
  float* O = r.F(r.S.O);
  float* Pd = r.F(r.S.Pd);
  float* Po = r.F(r.S.Po);
  float* Lf = r.F(r.S.Lf);
  float* Wf = r.F(r.S.Wf);
  const float* A = r.F(r.S.A);
  const float* Bm = r.F(r.S.Bm);
  const float* mi = r.F(r.S.misc);
  auto qproj = [&](int kk, int i) { return mi[(kk < r.T ? MS_QP : MS_QTP) + i]; };
  auto el = [&](const float* X, int i, int j) -> const float& { return X[(i * NX + j) * KB + kl]; };
  // D_k, O_k (rows r0, r0 + 1 of the thread's knot)
  if (r.act) {
    float qi[NX];
#pragma unroll
    for (int i = 0; i < NX; ++i) qi[i] = 1.f / qproj(k, i);
    if (k == 0) {
#pragma unroll
      for (int q = 0; q < kClRows; ++q)
#pragma unroll
        for (int j = 0; j < NX; ++j) {
          const int i = r.r0 + q;
          D[(i * NX + j) * KB + kl] = (i == j) ? qi[i] : 0.f;
          O[(i * NX + j) * KB + kl] = 0.f;
        }
    } else {
      float qt[NX], ri[NU];
#pragma unroll
      for (int i = 0; i < NX; ++i) qt[i] = 1.f / qproj(k - 1, i);
#pragma unroll
      for (int i = 0; i < NU; ++i) ri[i] = 1.f / mi[MS_RP + i];
#pragma unroll
      for (int q = 0; q < kClRows; ++q) {
        const int i = r.r0 + q;
#pragma unroll
        for (int j = 0; j < NX; ++j) {
          const int hi = i > j ? i : j, lo = i > j ? j : i;   // the lower-triangle order of stage_schur
          float sum = (hi == lo) ? qi[hi] : 0.f;
#pragma unroll
          for (int l = 0; l < NX; ++l) {
            const float ah = el(A, hi, l) - (hi == l ? 1.f : 0.f), al = el(A, lo, l) - (lo == l ? 1.f : 0.f);
            sum = fmaf(ah * qt[l], al, sum);
          }
#pragma unroll
          for (int l = 0; l < NU; ++l) sum = fmaf(Bm[(hi * NU + l) * KB + kl] * ri[l], Bm[(lo * NU + l) * KB + kl], sum);
          D[(i * NX + j) * KB + kl] = sum;
          O[(i * NX + j) * KB + kl] = (el(A, i, j) - (i == j ? 1.f : 0.f)) * qt[j];
        }
      }
    }
  }
  // O of the next CTA's first knot (block slot nk) from its staged A; zero without a next CTA
  // (Po there too: the last knot's rows read block slot nk against a zero halo vector)
  for (int e = r.tid; e < NX * NX; e += kClThreads) {
    const int i = e / NX, j = e % NX;
    O[e * KB + nk] = r.has_next ? (A[e * KB + nk] - (i == j ? 1.f : 0.f)) * (1.f / qproj(r.k0 + nk - 1, j)) : 0.f;
    if (!r.has_next) Po[e * KB + nk] = 0.f;
  }
  __syncthreads();
  // Pd_k = D_k^-1: Cholesky D = L L^T column by column (each thread its rows), W = L^-1 (each
  // thread its columns), D^-1 = W^T W (each thread its rows)
  bool fail = false;
#pragma unroll
  for (int j = 0; j < NX; ++j) {
    if (r.act) {
      float sd = el(D, j, j);
#pragma unroll
      for (int q = 0; q < j; ++q) sd -= el(Lf, j, q) * el(Lf, j, q);
      if (!(sd > 0.f)) { fail = true; sd = fabsf(el(D, j, j)) + 1e-30f; }
      const float d = sqrtf(sd);
      const float id = 1.f / d;
#pragma unroll
      for (int q2 = 0; q2 < kClRows; ++q2) {
        const int i = r.r0 + q2;
        if (i == j) Lf[(i * NX + j) * KB + kl] = d;
        if (i > j) {
          float t = el(D, i, j);
#pragma unroll
          for (int q = 0; q < j; ++q) t -= el(Lf, i, q) * el(Lf, j, q);
          Lf[(i * NX + j) * KB + kl] = t * id;
        }
      }
    }
    __syncthreads();
  }
  if (r.act && !fail) {
#pragma unroll
    for (int q2 = 0; q2 < kClRows; ++q2) {
      const int c = r.r0 + q2;   // this thread's columns of W
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        if (i < c) continue;
        float t = (i == c) ? 1.f : 0.f;
#pragma unroll
        for (int q = 0; q < NX; ++q)
          if (q >= c && q < i) t -= el(Lf, i, q) * el(Wf, q, c);
        Wf[(i * NX + c) * KB + kl] = t / el(Lf, i, i);
      }
    }
  }
  __syncthreads();
  if (r.act) {
#pragma unroll
    for (int q2 = 0; q2 < kClRows; ++q2) {
      const int i = r.r0 + q2;
#pragma unroll
      for (int j = 0; j < NX; ++j) {
        float v;
        if (fail) {
          v = (i == j) ? 1.f / (fabsf(el(D, i, i)) + 1e-30f) : 0.f;
        } else {
          const int hi = i > j ? i : j, lo = i > j ? j : i;
          float sum = 0.f;
#pragma unroll
          for (int q = 0; q < NX; ++q)
            if (q >= hi) sum += el(Wf, q, hi) * el(Wf, q, lo);
          v = sum;
        }
        Pd[(i * NX + j) * KB + kl] = v;
      }
    }
  }
  // the previous CTA's last Pd, for this CTA's first Po
  cl_release_barrier<M>(r);
  if (r.has_prev && !r.broken) {
    const uint32_t base = r.remote(r.S.Pd, r.rank - 1);
    for (int e = r.tid; e < NX * NX; e += kClThreads)
      r.F(r.S.pdp)[e] = cl::ld_f32(base + 4u * (uint32_t)(e * KB + r.KC - 1));
  }
  __syncthreads();
  // Po_k = -Pd_k (O_k Pd_{k-1}): t1 rows into the Cholesky scratch, then Po rows
  if (r.act && k > 0) {
#pragma unroll
    for (int q2 = 0; q2 < kClRows; ++q2) {
      const int i = r.r0 + q2;
#pragma unroll
      for (int j = 0; j < NX; ++j) {
        float sum = 0.f;
#pragma unroll
        for (int l = 0; l < NX; ++l) {
          const float pp = (kl == 0) ? r.F(r.S.pdp)[l * NX + j] : Pd[(l * NX + j) * KB + kl - 1];
          sum = fmaf(el(O, i, l), pp, sum);
        }
        Lf[(i * NX + j) * KB + kl] = sum;
      }
    }
  }
  __syncthreads();
  if (r.act) {
#pragma unroll
    for (int q2 = 0; q2 < kClRows; ++q2) {
      const int i = r.r0 + q2;
#pragma unroll
      for (int j = 0; j < NX; ++j) {
        float sum = 0.f;
        if (k > 0) {
#pragma unroll
          for (int l = 0; l < NX; ++l) sum = fmaf(el(Pd, i, l), el(Lf, l, j), sum);
        }
        Po[(i * NX + j) * KB + kl] = k > 0 ? -sum : 0.f;
      }
    }
  }
  // the next CTA's first Po (block slot nk)
  cl_release_barrier<M>(r);
  if (r.has_next && !r.broken) {
    const uint32_t base = r.remote(r.S.Po, r.rank + 1);
    for (int e = r.tid; e < NX * NX; e += kClThreads) Po[e * KB + nk] = cl::ld_f32(base + 4u * (uint32_t)(e * KB));
  }
  __syncthreads();
  return __syncthreads_or(fail && r.act) != 0;
}

struct ClSync {
  int phase;
  bool broken;
};

// r is taken by value (so that the caller's copy stays in registers); returns its all-reduce
// state after the call.
template <class M>
__device__ __noinline__ ClSync cl_hp_residual(ClRun<M> r, bool push_lp, int rb) {
  constexpr int NX = M::NX, NU = M::NU;
  const int KB = r.S.KB, KV = r.S.KV, kl = r.kl, s = kl + 1;
  const int k = r.k0 + kl;
  double* LP = r.Dd(r.S.LP);
  double* WX = r.Dd(r.S.WX);
  double* WU = r.Dd(r.S.WU);
  const double* G = r.Dd(r.S.G);
  const float* A = r.F(r.S.A);
  const float* Bm = r.F(r.S.Bm);
  if (push_lp) {
    if (r.act && kl == 0 && r.has_prev && !r.broken) {
      const uint32_t q = r.rank - 1, rbar = r.red_bar(q);
#pragma unroll
      for (int j = 0; j < kClRows; ++j) {
        const int i = r.r0 + j;
        cl::st_async_f64(r.remote_d(r.S.LP + i * KV + r.KC + 1, q), LP[i * KV + s], rbar);
      }
    }
    cl_barrier<M>(r, r.has_next ? 8u * NX : 0u);
  }
  // pass 1: w = H^T LP at knot k (A_k, B_k at block slot kl + 1, stored as A_k + I)
  if (r.act) {
    double ln[NX];
#pragma unroll
    for (int j = 0; j < NX; ++j) ln[j] = (k < r.T) ? LP[j * KV + s + 1] : 0.0;
    const bool send = kl == r.nk - 1 && r.has_next && !r.broken;
    const uint32_t q = r.rank + 1, rbar = send ? r.red_bar(q) : 0u;
#pragma unroll
    for (int j = 0; j < kClRows; ++j) {
      const int i = r.r0 + j;
      double acc = LP[i * KV + s];
      if (k < r.T) {
        acc -= ln[i];
#pragma unroll
        for (int c = 0; c < NX; ++c) acc += (double)A[(c * NX + i) * KB + kl + 1] * ln[c];
      }
      WX[i * KV + s] = acc;
      if (send) cl::st_async_f64(r.remote_d(r.S.WX + i * KV + 0, q), acc, rbar);
    }
    for (int u = r.r0 / kClRows; u < NU; u += r.RG) {
      double acc = 0.0;
      if (k < r.T) {
#pragma unroll
        for (int c = 0; c < NX; ++c) acc += (double)Bm[(c * NU + u) * KB + kl + 1] * ln[c];
      }
      WU[u * KV + s] = acc;
      if (send) cl::st_async_f64(r.remote_d(r.S.WU + u * KV + 0, q), acc, rbar);
    }
  }
  cl_barrier<M>(r, r.has_prev ? 8u * (NX + NU) : 0u);
  // pass 2: (H G^-1 w)_k on this thread's rows, then R = gamma - that
  if (r.act) {
    float rv[kClRows], zero[kClRows];
    double vx[NX], vu[NU];
    if (k > 0) {
#pragma unroll
      for (int j = 0; j < NX; ++j) vx[j] = WX[j * KV + s - 1] * r.qinv(k - 1, j);
#pragma unroll
      for (int j = 0; j < NU; ++j) vu[j] = WU[j * KV + s - 1] * r.rinv(j);
    }
#pragma unroll
    for (int j = 0; j < kClRows; ++j) {
      const int i = r.r0 + j;
      double acc = WX[i * KV + s] * r.qinv(k, i);
      if (k > 0) {
        acc -= vx[i];
#pragma unroll
        for (int c = 0; c < NX; ++c) acc += (double)A[(i * NX + c) * KB + kl] * vx[c];
#pragma unroll
        for (int c = 0; c < NU; ++c) acc += (double)Bm[(i * NU + c) * KB + kl] * vu[c];
      }
      rv[j] = (float)(G[i * KV + s] - acc);
      r.F(r.S.R[rb])[i * KV + s] = rv[j];
      zero[j] = 0.f;
    }
    cl_push_pair<M>(r, r.S.rh, r.S.yh, rv, zero);
  }
  cl_barrier<M>(r, r.halo_bytes(8u * NX));
  return ClSync{r.phase, r.broken};
}

template <class M>
__device__ __forceinline__ void cl_true_residual(ClRun<M>& r, bool push_lp, int rb) {
  const ClSync st = cl_hp_residual<M>(r, push_lp, rb);
  r.phase = st.phase;
  r.broken = st.broken;
}

// ---- double-float rescue on the cluster (stage_pcg_df distributed) ------------------------

// Sum a double-float value over the cluster: warp butterflies and warp partials with df_add,
// then every CTA's partial into a slot of every CTA (st.async of its two floats), summed in rank
// order; bitwise the same total everywhere.  halo_rx as in cl_sum.
template <class M>
__device__ __forceinline__ dfl cl_sum_df(ClRun<M>& r, dfl v, uint32_t halo_rx) {
  v = df_warp_sum(v);
  const int b = r.phase & 1;
  const uint32_t par = (uint32_t)(r.phase >> 1) & 1u;
  float* wp = r.F(r.S.wpart) + b * (kClThreads / 32) * kClNV;
  float* sl = r.F(r.S.slots) + b * kClMaxCtas * kClNV;
  if ((r.tid & 31) == 0) { wp[(r.tid >> 5) * kClNV] = v.hi; wp[(r.tid >> 5) * kClNV + 1] = v.lo; }
  __syncthreads();
  if (r.tid < (int)r.ncta && !r.broken) {
    dfl t = {wp[0], wp[1]};
    for (int q = 1; q < kClThreads / 32; ++q) t = df_add(t, dfl{wp[q * kClNV], wp[q * kClNV + 1]});
    const uint32_t dst = r.remote(r.S.slots + b * kClMaxCtas * kClNV + (int)r.rank * kClNV, (uint32_t)r.tid);
    const uint32_t rb = r.red_bar((uint32_t)r.tid);
    cl::st_async_f32(dst, t.hi, rb);
    cl::st_async_f32(dst + 4u, t.lo, rb);
  }
  if (r.tid == 0 && !r.broken) cl::arrive_expect_tx(r.bar(b), r.ncta * 8u + halo_rx);
  bool ok = r.broken ? false : cl::wait(r.bar(b), par, kClWaitNs);
  ok = __syncthreads_and(ok) != 0;
  if (!ok) r.broken = true;
  dfl t = {sl[0], sl[1]};
  for (uint32_t q = 1; q < r.ncta; ++q) t = df_add(t, dfl{sl[q * kClNV], sl[q * kClNV + 1]});
  ++r.phase;
  return t;
}

// Send this thread's rows of a boundary knot's double-float values (a, b) into the df staging
// arrays of the neighbours (side 1 of the previous CTA, side 0 of the next) for the coming phase.
template <class M>
__device__ __forceinline__ void cl_push_df(ClRun<M>& r, int st_a, int st_b, const dfl* a, const dfl* b) {
  constexpr int NX = M::NX;
  if (!r.act || r.broken) return;
  auto send = [&](uint32_t q, int side) {
    const uint32_t rb = r.red_bar(q);
    const uint32_t da = r.remote(st_a + 2 * (side * NX + r.r0), q), db = r.remote(st_b + 2 * (side * NX + r.r0), q);
#pragma unroll
    for (int i = 0; i < kClRows; ++i) {
      cl::st_async_f32(da + 8u * i, a[i].hi, rb);
      cl::st_async_f32(da + 8u * i + 4u, a[i].lo, rb);
      cl::st_async_f32(db + 8u * i, b[i].hi, rb);
      cl::st_async_f32(db + 8u * i + 4u, b[i].lo, rb);
    }
  };
  if (r.kl == 0 && r.has_prev) send(r.rank - 1, 1);
  if (r.kl == r.nk - 1 && r.has_next) send(r.rank + 1, 0);
}

// halo slots of the df vector `v` (slot 0 from side 0, slot nk + 1 from side 1) = a + s b from
// the df staging
template <class M>
__device__ __forceinline__ void cl_halo_df(ClRun<M>& r, dfl* v, int st_a, int st_b, dfl sc) {
  constexpr int NX = M::NX;
  if (r.tid < 2 * NX) {
    const int side = r.tid / NX, i = r.tid % NX;
    if (side == 0 ? r.has_prev : r.has_next) {
      const dfl* ha = reinterpret_cast<const dfl*>(r.F(st_a));
      const dfl* hb = reinterpret_cast<const dfl*>(r.F(st_b));
      v[i * r.S.KV + (side == 0 ? 0 : r.nk + 1)] = df_add(ha[side * NX + i], df_mul(sc, hb[side * NX + i]));
    }
  }
  __syncthreads();
}

// out = S v (= H G^-1 H^T v) on the own knots in double-float from the FP32 factors and the
// reciprocal weights (df_apply distributed): v needs its next-CTA halo slot; one phase inside
// (the previous CTA's last H^T v).
template <class M>
__device__ __forceinline__ void cl_df_apply(ClRun<M>& r, const dfl* v, dfl* out, const dfl (&qx)[M::NX],
                                            const dfl (&qT)[M::NX], const dfl (&ri)[M::NU]) {
  constexpr int NX = M::NX, NU = M::NU;
  const int KB = r.S.KB, KV = r.S.KV, kl = r.kl, sl = kl + 1, k = r.k0 + kl;
  const float* A = r.F(r.S.A);
  const float* Bm = r.F(r.S.Bm);
  dfl* WX = reinterpret_cast<dfl*>(r.F(r.S.dWX));
  dfl* WU = reinterpret_cast<dfl*>(r.F(r.S.dWU));
  if (r.act) {
    const bool send = kl == r.nk - 1 && r.has_next && !r.broken;
    const uint32_t q = r.rank + 1, rbar = send ? r.red_bar(q) : 0u;
#pragma unroll
    for (int j = 0; j < kClRows; ++j) {
      const int i = r.r0 + j;
      dacc a = dacc_zero();
      dacc_add(a, v[i * KV + sl]);
      if (k < r.T) {   // (A_k + I)^T v_{k+1} - v_{k+1}
#pragma unroll
        for (int c = 0; c < NX; ++c) dacc_fma(a, A[(c * NX + i) * KB + kl + 1], v[c * KV + sl + 1]);
        dacc_add(a, df_neg(v[i * KV + sl + 1]));
      }
      const dfl w = dacc_get(a);
      WX[i * KV + sl] = w;
      if (send) {
        const uint32_t d = r.remote(r.S.dWX + 2 * (i * KV + 0), q);
        cl::st_async_f32(d, w.hi, rbar);
        cl::st_async_f32(d + 4u, w.lo, rbar);
      }
    }
    for (int u = r.r0 / kClRows; u < NU; u += r.RG) {
      dacc a = dacc_zero();
      if (k < r.T) {
#pragma unroll
        for (int c = 0; c < NX; ++c) dacc_fma(a, Bm[(c * NU + u) * KB + kl + 1], v[c * KV + sl + 1]);
      }
      const dfl w = dacc_get(a);
      WU[u * KV + sl] = w;
      if (send) {
        const uint32_t d = r.remote(r.S.dWU + 2 * (u * KV + 0), q);
        cl::st_async_f32(d, w.hi, rbar);
        cl::st_async_f32(d + 4u, w.lo, rbar);
      }
    }
  }
  cl_barrier<M>(r, r.has_prev ? 8u * (NX + NU) : 0u);
  if (r.act) {
    dfl vx[NX], vu[NU];
    if (k > 0) {
#pragma unroll
      for (int j = 0; j < NX; ++j) vx[j] = df_mul(WX[j * KV + sl - 1], qx[j]);   // k - 1 < T
#pragma unroll
      for (int j = 0; j < NU; ++j) vu[j] = df_mul(WU[j * KV + sl - 1], ri[j]);
    }
#pragma unroll
    for (int j = 0; j < kClRows; ++j) {
      const int i = r.r0 + j;
      dacc a = dacc_zero();
      dacc_add(a, df_mul(WX[i * KV + sl], k < r.T ? qx[i] : qT[i]));
      if (k > 0) {
#pragma unroll
        for (int c = 0; c < NX; ++c) dacc_fma(a, A[(i * NX + c) * KB + kl], vx[c]);
        dacc_add(a, df_neg(vx[i]));
#pragma unroll
        for (int c = 0; c < NU; ++c) dacc_fma(a, Bm[(i * NU + c) * KB + kl], vu[c]);
      }
      out[i * KV + sl] = dacc_get(a);
    }
  }
}

// Rows of z = Phi^-1 v in double-float (FP32 blocks, compensated accumulation); v needs both halo
// slots.
template <class M>
__device__ __forceinline__ void cl_precond_df(const ClRun<M>& r, const dfl* v, dfl (&z)[kClRows]) {
  constexpr int NX = M::NX;
  const int KB = r.S.KB, KV = r.S.KV, kl = r.kl, sl = kl + 1;
  const float* Pd = r.F(r.S.Pd);
  const float* Po = r.F(r.S.Po);
#pragma unroll
  for (int q = 0; q < kClRows; ++q) {
    const int i = r.r0 + q;
    dacc a = dacc_zero();
#pragma unroll
    for (int j = 0; j < NX; ++j) dacc_fma(a, Pd[(i * NX + j) * KB + kl], v[j * KV + sl]);
#pragma unroll
    for (int j = 0; j < NX; ++j) dacc_fma(a, Po[(i * NX + j) * KB + kl], v[j * KV + sl - 1]);
#pragma unroll
    for (int j = 0; j < NX; ++j) dacc_fma(a, Po[(j * NX + i) * KB + kl + 1], v[j * KV + sl + 1]);
    z[q] = dacc_get(a);
  }
}

struct ClDfOut {
  int phase, it;
  bool broken, converged, breakdown;
};

// The double-float rescue of one solve on the cluster (stage_pcg_df's iteration with every
// vector in shared memory): continues from the FP64 solution LP; on return LP holds the result
// (the caller then forms the FP64 true residual and H^T LP).  Three phases per iteration (the
// operator's halo, p^T S p with the r, S p halos, r^T z with the z, p halos).
template <class M>
__device__ __noinline__ ClDfOut cl_pcg_df(ClRun<M> r, float eta0f, int maxit, float tol) {
  constexpr int NX = M::NX, NU = M::NU;
  const int KV = r.S.KV, sl = r.kl + 1;
  ClDfOut out{0, 0, false, false, false};
  dfl* X = reinterpret_cast<dfl*>(r.F(r.S.dX));
  dfl* R = reinterpret_cast<dfl*>(r.F(r.S.dR));
  dfl* Pv = reinterpret_cast<dfl*>(r.F(r.S.dP));
  dfl* Y = reinterpret_cast<dfl*>(r.F(r.S.dY));
  dfl* Z = reinterpret_cast<dfl*>(r.F(r.S.dZ));
  double* LP = r.Dd(r.S.LP);
  const double* G = r.Dd(r.S.G);
  dfl qx[NX], qT[NX], ri[NU];
#pragma unroll
  for (int i = 0; i < NX; ++i) { qx[i] = df_from(r.qinv(0, i)); qT[i] = df_from(r.qinv(r.T, i)); }
#pragma unroll
  for (int i = 0; i < NU; ++i) ri[i] = df_from(r.rinv(i));
  const dfl thr = df_mulf(df_make(eta0f), tol * tol);
  const dfl zero = {0.f, 0.f};
  const uint32_t pair_rx = r.halo_bytes(16u * NX);   // two df vectors of NX from each neighbour
  for (int idx = r.tid; idx < NX * KV; idx += kClThreads) {
    X[idx] = zero; R[idx] = zero; Pv[idx] = zero; Y[idx] = zero; Z[idx] = zero;
  }
  for (int idx = r.tid; idx < 16 * NX; idx += kClThreads) r.sm[r.S.drh + idx] = 0.f;   // the four stagings
  __syncthreads();
  dfl xr[kClRows];
  if (r.act) {
#pragma unroll
    for (int q = 0; q < kClRows; ++q) { xr[q] = df_from(LP[(r.r0 + q) * KV + sl]); X[(r.r0 + q) * KV + sl] = xr[q]; }
  }
  // X's next-CTA halo (the previous CTA receives this CTA's first knot), then R = gamma - S X
  cl_push_df<M>(r, r.S.dzh, r.S.dph, xr, xr);
  cl_barrier<M>(r, r.halo_bytes(16u * NX));
  cl_halo_df<M>(r, X, r.S.dzh, r.S.dzh, zero);
  cl_df_apply<M>(r, X, Y, qx, qT, ri);
  dfl rr[kClRows], zr[kClRows];
  if (r.act) {
#pragma unroll
    for (int q = 0; q < kClRows; ++q) {
      const int i = r.r0 + q;
      rr[q] = df_sub(df_from(G[i * KV + sl]), Y[i * KV + sl]);
      R[i * KV + sl] = rr[q];
    }
  }
  cl_push_df<M>(r, r.S.drh, r.S.dyh, rr, rr);
  cl_barrier<M>(r, pair_rx);
  cl_halo_df<M>(r, R, r.S.drh, r.S.drh, zero);
  // z = Phi^-1 r, p = z, eta = r^T z
  dacc ea = dacc_zero();
  if (r.act) {
    cl_precond_df<M>(r, R, zr);
#pragma unroll
    for (int q = 0; q < kClRows; ++q) {
      const int i = r.r0 + q;
      Z[i * KV + sl] = zr[q];
      Pv[i * KV + sl] = zr[q];
      dacc_fma(ea, rr[q], zr[q]);
    }
  }
  cl_push_df<M>(r, r.S.dzh, r.S.dph, zr, zr);
  dfl eta = cl_sum_df<M>(r, dacc_get(ea), pair_rx);
  cl_halo_df<M>(r, Pv, r.S.dzh, r.S.dzh, zero);
  int it = 0;
  bool converged = !(eta.hi > thr.hi);
  while (!converged && it < maxit && !r.broken) {
    // y = S p, v = p^T y; boundary knots send r and y
    cl_df_apply<M>(r, Pv, Y, qx, qT, ri);
    dacc va = dacc_zero();
    dfl yr[kClRows], pr[kClRows];
    if (r.act) {
#pragma unroll
      for (int q = 0; q < kClRows; ++q) {
        const int i = r.r0 + q;
        yr[q] = Y[i * KV + sl];
        rr[q] = R[i * KV + sl];
        pr[q] = Pv[i * KV + sl];
        dacc_fma(va, pr[q], yr[q]);
      }
    }
    cl_push_df<M>(r, r.S.drh, r.S.dyh, rr, yr);
    const dfl v = cl_sum_df<M>(r, dacc_get(va), pair_rx);
    if (!(v.hi > 0.f) || !isfinite(v.hi)) { out.breakdown = true; break; }
    const dfl alpha = df_div(eta, v);
    // x += alpha p, r -= alpha y; r's halos from the neighbours' old r and y
    if (r.act) {
#pragma unroll
      for (int q = 0; q < kClRows; ++q) {
        const int i = r.r0 + q;
        X[i * KV + sl] = df_add(X[i * KV + sl], df_mul(alpha, pr[q]));
        rr[q] = df_sub(rr[q], df_mul(alpha, yr[q]));
        R[i * KV + sl] = rr[q];
      }
    }
    cl_halo_df<M>(r, R, r.S.drh, r.S.dyh, df_neg(alpha));
    // z = Phi^-1 r, eta = r^T z; boundary knots send z and the old p
    dacc na = dacc_zero();
    if (r.act) {
      cl_precond_df<M>(r, R, zr);
#pragma unroll
      for (int q = 0; q < kClRows; ++q) {
        Z[(r.r0 + q) * KV + sl] = zr[q];
        dacc_fma(na, rr[q], zr[q]);
      }
    }
    cl_push_df<M>(r, r.S.dzh, r.S.dph, zr, pr);
    const dfl eta_new = cl_sum_df<M>(r, dacc_get(na), pair_rx);
    ++it;
    if (!(eta_new.hi > thr.hi)) { converged = true; break; }
    if (!isfinite(eta_new.hi)) break;
    const dfl beta = df_div(eta_new, eta);
    eta = eta_new;
    // p = z + beta p (own rows and the next CTA's halo from its z and old p)
    if (r.act) {
#pragma unroll
      for (int q = 0; q < kClRows; ++q) {
        const int i = r.r0 + q;
        Pv[i * KV + sl] = df_add(zr[q], df_mul(beta, pr[q]));
      }
    }
    cl_halo_df<M>(r, Pv, r.S.dzh, r.S.dph, beta);
  }
  if (r.act) {
#pragma unroll
    for (int q = 0; q < kClRows; ++q) LP[(r.r0 + q) * KV + sl] = df_to(X[(r.r0 + q) * KV + sl]);
  }
  out.phase = r.phase;
  out.broken = r.broken;
  out.it = it;
  out.converged = converged;
  return out;
}

struct ClResult {
  int it;
  bool converged;
  float eta0;
  bool chol_fail;   // a diagonal Schur block failed Cholesky (formed blocks only)
  int df_it;        // iterations of the double-float rescue (0 when FP32 converged)
  bool df_breakdown;
  bool df_converged;
};

// The distributed PCG of one OCP, run by every CTA of the cluster.  ws: the OCP's global
// workspace (leader's layout L).  On return LP (the solution) and WX, WU (= H^T LP) are back in
// the global workspace.
// State of a CTA after a stage of the solve: the all-reduce counters and the result so far.
struct ClStage {
  int phase;
  uint32_t rel_par;
  bool broken;
  int rb;
  ClResult res;
};

template <class M>
__device__ __noinline__ ClStage cl_pcg_fp32(ClRun<M> r, const KParams& P, float* ws, bool form);
template <class M>
__device__ __noinline__ ClStage cl_pcg_finish(ClRun<M> r, const KParams& P, float* ws, ClStage st);

// One solve on the cluster, in stages that each take the CTA's state by value (so every stage
// keeps it in registers): the FP32 iteration, the double-float rescue when that stagnated, and the
// write-back.  form: the S and Phi^-1 blocks are formed here from the factors (and written to the
// global workspace), else they are read from it.
template <class M>
__device__ __forceinline__ ClResult cl_pcg(ClRun<M>& rin, const KParams& P, int K, int T, float* ws, bool form) {
  rin.bind(K, T);
  ClStage st = cl_pcg_fp32<M>(rin, P, ws, form);
  rin.phase = st.phase;
  rin.rel_par = st.rel_par;
  rin.broken = st.broken;
  if (!st.res.converged && !rin.broken) {
    const ClDfOut d = cl_pcg_df<M>(rin, st.res.eta0, P.opt.pcg_max_iters, P.opt.pcg_tol);
    rin.phase = d.phase;
    rin.broken = d.broken;
    st.res.df_it = d.it;
    st.res.df_breakdown = d.breakdown;
    st.res.df_converged = d.converged;
    if (!rin.broken) {
      const ClSync sy = cl_hp_residual<M>(rin, true, st.rb);
      rin.phase = sy.phase;
      rin.broken = sy.broken;
    }
  }
  st.phase = rin.phase;
  st.broken = rin.broken;
  st = cl_pcg_finish<M>(rin, P, ws, st);
  rin.phase = st.phase;
  rin.rel_par = st.rel_par;
  rin.broken = st.broken;
  return st.res;
}

template <class M>
__device__ __noinline__ ClStage cl_pcg_fp32(ClRun<M> r, const KParams& P, float* ws, bool form) {
  constexpr int NX = M::NX, NU = M::NU;
  const int K = r.K;
  ClResult res{0, false, 0.f, false, 0, false, false};
  const Layout L = make_layout(NX, NU, K, kClThreads, P.opt.exact_hessian, 0);
  const int KP = L.KP, KB = r.S.KB, KV = r.S.KV, nk = r.nk, k0 = r.k0;
  const double* wd = reinterpret_cast<const double*>(ws);
  // stage the blocks (own knots and the next CTA's first knot) and vectors from global memory;
  // missing neighbours and the unused slot-0 blocks (O_0, Phi^-1 off-diagonal, A, B at k = 0)
  // are zero
  {
    const int nb = nk + 1;
    const int offs[5] = {L.A, L.D, L.O, L.Pd, L.Po};
    const int so[5] = {r.S.A, r.S.D, r.S.O, r.S.Pd, r.S.Po};
    for (int a = 0; a < (form ? 1 : 5); ++a) {
      for (int idx = r.tid; idx < NX * NX * nb; idx += kClThreads) {
        const int e = idx / nb, j = idx % nb, k = k0 + j;
        const bool zero_at0 = (a == 0 || a == 2 || a == 4) && k == 0;
        r.sm[so[a] + e * KB + j] = (nk > 0 && k < K && !zero_at0) ? __ldcg(ws + offs[a] + e * KP + k) : 0.f;
      }
    }
    for (int idx = r.tid; idx < NX * NU * nb; idx += kClThreads) {
      const int e = idx / nb, j = idx % nb, k = k0 + j;
      r.sm[r.S.Bm + e * KB + j] = (nk > 0 && k < K && k > 0) ? __ldcg(ws + L.Bm + e * KP + k) : 0.f;
    }
    for (int idx = r.tid; idx < NX * KV; idx += kClThreads) {
      const int i = idx / KV, sl = idx % KV, k = k0 + sl - 1;
      const bool in = nk > 0 && sl <= nk + 1 && k >= 0 && k < K;
      r.Dd(r.S.LP)[idx] = in ? __ldcg(wd + L.d_lamp + i * KP + k) : 0.0;
      r.Dd(r.S.G)[idx] = in ? __ldcg(wd + L.d_gam + i * KP + k) : 0.0;
      r.Dd(r.S.WX)[idx] = 0.0;
      r.F(r.S.Pv[0])[idx] = 0.f;
      r.F(r.S.Pv[1])[idx] = 0.f;
      r.F(r.S.R[0])[idx] = 0.f;
      r.F(r.S.R[1])[idx] = 0.f;
      r.F(r.S.Y)[idx] = 0.f;
      r.F(r.S.Z)[idx] = 0.f;
      r.F(r.S.DL)[idx] = 0.f;
    }
    for (int idx = r.tid; idx < NU * KV; idx += kClThreads) r.Dd(r.S.WU)[idx] = 0.0;
    for (int idx = r.tid; idx < kMisc; idx += kClThreads) r.sm[r.S.misc + idx] = __ldcg(ws + L.misc + idx);
    for (int idx = r.tid; idx < 8 * NX; idx += kClThreads) r.sm[r.S.rh + idx] = 0.f;  // rh, yh, zh, ph
  }
  __syncthreads();
  bool chol_fail = false;
  if (form) {
    chol_fail = cl_form_blocks<M>(r);
    // the formed blocks of the own knots back to the global workspace (rescue, inspect)
    const int offs[4] = {L.D, L.O, L.Pd, L.Po};
    const int so[4] = {r.S.D, r.S.O, r.S.Pd, r.S.Po};
    for (int a = 0; a < 4; ++a)
      for (int idx = r.tid; idx < NX * NX * nk; idx += kClThreads) {
        const int e = idx / nk, j = idx % nk;
        ws[offs[a] + e * KP + k0 + j] = r.sm[so[a] + e * KB + j];
      }
  }
  const float tol2 = P.opt.pcg_tol * P.opt.pcg_tol;
  const float dl2 = P.opt.ru_delta * P.opt.ru_delta;
  const int maxit = P.opt.pcg_max_iters;
  const uint32_t pair_rx = r.halo_bytes(8u * NX);  // two vectors of NX floats from each neighbour
  double* LP = r.Dd(r.S.LP);
  float* DL = r.F(r.S.DL);
  const int s = r.kl + 1;
  int pb = 0, rb = 0;  // current buffers of p (holds the previous p until the next step) and r

  // true residual of the initial guess (its next-CTA LP halo came from global memory), z, eta,
  // eta_0 = gamma^T Phi^-1 gamma from the FP32-rounded gamma
  cl_true_residual<M>(r, false, rb);
  float e0[3] = {0.f, 0.f, 0.f};
  e0[0] = cl_step_pc<M, false>(r, rb, rb, pb, 0.f);
  if (r.tid == 0 && chol_fail) e0[2] = 1.f;
  if (r.act) {
    float gm[NX], gc[NX], gp[NX], gt[kClRows];
    const double* G = r.Dd(r.S.G);
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      gm[j] = (float)G[j * KV + s - 1];
      gc[j] = (float)G[j * KV + s];
      gp[j] = (float)G[j * KV + s + 1];
    }
    cl_block_rows<M>(r, r.S.Pd, r.S.Po, gm, gc, gp, gt);
#pragma unroll
    for (int q = 0; q < kClRows; ++q) e0[1] = fmaf(gc[r.r0 + q], gt[q], e0[1]);
  }
  cl_sum<M, 3>(r, e0, pair_rx);
  float eta = e0[0];
  const float eta0 = e0[1];
  res.eta0 = eta0;
  res.chol_fail = e0[2] > 0.f;
  float beta = 0.f;  // p = z for the first direction (the old p is zero)
  float eta_ref = eta, eta_true = eta;
  int it = 0, stall = 0;
  bool converged = !(eta > tol2 * eta0);
  bool folded = true;
  while (!converged && it < maxit && !r.broken) {
    // y = S p, v = p^T y
    float v[1] = {cl_step_sp<M>(r, pb, pb ^ 1, rb, beta)};
    pb ^= 1;
    cl_sum<M, 1>(r, v, pair_rx);
    if (!(v[0] > 0.f) || !isfinite(v[0])) break;
    const float alpha = eta / v[0];
    // r -= alpha y, dl += alpha p, z = Phi^-1 r, eta = r^T z
    float e1[1] = {cl_step_pc<M, true>(r, rb, rb ^ 1, pb, alpha)};
    rb ^= 1;
    folded = false;
    cl_sum<M, 1>(r, e1, pair_rx);
    float eta_new = e1[0];
    ++it;
    if (eta_new < dl2 * eta_ref || !(eta_new > tol2 * eta0) || it >= maxit || !isfinite(eta_new)) {
      // reliable update: fold the FP32 correction into the FP64 solution, true residual
      if (r.act) {
#pragma unroll
        for (int q = 0; q < kClRows; ++q) {
          const int i = r.r0 + q;
          LP[i * KV + s] += (double)DL[i * KV + s];
          DL[i * KV + s] = 0.f;
        }
      }
      folded = true;
      cl_true_residual<M>(r, true, rb);
      float e2[1] = {cl_step_pc<M, false>(r, rb, rb, pb, 0.f)};
      cl_sum<M, 1>(r, e2, pair_rx);
      eta_new = e2[0];
      eta_ref = eta_new;
      if (!(eta_new > tol2 * eta0)) { converged = true; break; }
      if (!isfinite(eta_new)) break;
      if (eta_new > 0.25f * eta_true) {
        if (++stall >= 2) break;
      } else {
        stall = 0;
      }
      eta_true = eta_new;
      if (it >= maxit) break;
    }
    beta = eta_new / eta;
    eta = eta_new;
  }
  if (!folded && !r.broken) {
    if (r.act) {
#pragma unroll
      for (int q = 0; q < kClRows; ++q) {
        const int i = r.r0 + q;
        LP[i * KV + s] += (double)DL[i * KV + s];
      }
    }
    cl_true_residual<M>(r, true, rb);
  }
  res.it = it;
  res.converged = converged && !r.broken;
  return ClStage{r.phase, r.rel_par, r.broken, rb, res};
}

// Own knots of LP, WX, WU back to the global workspace, then a release barrier over the cluster.
template <class M>
__device__ __noinline__ ClStage cl_pcg_finish(ClRun<M> r, const KParams& P, float* ws, ClStage st) {
  constexpr int NX = M::NX, NU = M::NU;
  r.phase = st.phase;
  r.rel_par = st.rel_par;
  r.broken = st.broken;
  const Layout L = make_layout(NX, NU, r.K, kClThreads, P.opt.exact_hessian, 0);
  const int KP = L.KP, KV = r.S.KV, nk = r.nk, k0 = r.k0;
  double* LP = r.Dd(r.S.LP);
  // own knots of LP, WX, WU back to the global workspace
  if (!r.broken) {
    double* gd = reinterpret_cast<double*>(ws);
    for (int idx = r.tid; idx < NX * nk; idx += kClThreads) {
      const int i = idx / nk, j = idx % nk;
      gd[L.d_lamp + i * KP + k0 + j] = LP[i * KV + j + 1];
      gd[L.d_wx + i * KP + k0 + j] = r.Dd(r.S.WX)[i * KV + j + 1];
    }
    for (int idx = r.tid; idx < NU * nk; idx += kClThreads) {
      const int i = idx / nk, j = idx % nk;
      gd[L.d_wu + i * KP + k0 + j] = r.Dd(r.S.WU)[i * KV + j + 1];
    }
  }
  cl_release_barrier<M>(r);
  st.phase = r.phase;
  st.rel_par = r.rel_par;
  st.broken = r.broken;
  return st;
}

// Leader: send a command to the other CTAs of the cluster.  The team's earlier global-memory
// writes are released with it.
template <class M>
__device__ void cl_command(ClRun<M>& r, int cmd, int ocp, int K, int T, int form) {
  __syncthreads();
  if (r.tid == 0) {
    int* job = reinterpret_cast<int*>(r.sm + r.S.job);
    job[0] = cmd; job[1] = ocp; job[2] = K; job[3] = T; job[4] = form;
  }
  __syncthreads();
  if (r.tid >= 1 && r.tid < (int)r.ncta && !r.broken) cl::arrive_remote(cl::map(r.bar(CB_CMD), (uint32_t)r.tid));
}

// Other CTAs: run the leader's PCG commands until it sends CL_EXIT (or a wait runs out).
template <class M>
__device__ void cl_follower(ClRun<M>& r, const KParams& P, float* ws) {
  while (!r.broken) {
    bool ok = true;
    if (r.tid == 0) ok = cl::wait(r.bar(CB_CMD), r.cmd_par, kClWaitNs);
    ok = __syncthreads_and(ok) != 0;
    if (!ok) { r.broken = true; break; }
    r.cmd_par ^= 1u;
    const uint32_t jb = r.remote(r.S.job, 0);
    const int cmd = cl::ld_s32(jb), K = cl::ld_s32(jb + 8), T = cl::ld_s32(jb + 12), form = cl::ld_s32(jb + 16);
    if (cmd != CL_PCG) break;
    cl_pcg<M>(r, P, K, T, ws, form != 0);
  }
}

}  // namespace dmpc
