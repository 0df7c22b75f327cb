// a4 distributed over a thread-block cluster: Algorithm 4 for one OCP whose workspace does not
// fit in one CTA's shared memory (12-state rigid body, T up to a few hundred).  CTA 0 of the
// cluster (the leader) runs every other stage of the SQP iteration and the backward pass from the
// OCP's global-memory workspace, as the single-team kernel does.  At each PCG solve it hands the
// solve to all CTAs of the cluster: CTA r copies the knots [r KC, (r+1) KC) of the S and Phi^-1
// blocks, the factors A_t, B_t and the FP64 vectors into its own shared memory, and the PCG then
// runs with every block resident on chip:
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
//     factors (hp_apply's two passes, distributed the same way) and the stagnation test hands
//     the solve back to the leader, which finishes it with the double-float rescue from global
//     memory, exactly as the single-team kernel does.
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
  S.Lf = f; f += nx * nx * S.KB;
  S.Wf = f; f += nx * nx * S.KB;
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

struct ClResult {
  int it;
  bool converged;
  float eta0;
  bool chol_fail;   // a diagonal Schur block failed Cholesky (formed blocks only)
};

// The distributed PCG of one OCP, run by every CTA of the cluster.  ws: the OCP's global
// workspace (leader's layout L).  On return LP (the solution) and WX, WU (= H^T LP) are back in
// the global workspace.
template <class M>
__device__ __forceinline__ ClResult cl_pcg_body(ClRun<M>& r, const KParams& P, int K, int T, float* ws, bool form);

// Works on a register copy of the CTA's state and writes back what the solve changed.  form: the
// S and Phi^-1 blocks are formed here from the factors (and written to the global workspace),
// else they are read from it.
template <class M>
__device__ __forceinline__ ClResult cl_pcg(ClRun<M>& rin, const KParams& P, int K, int T, float* ws, bool form) {
  ClRun<M> r = rin;
  const ClResult res = cl_pcg_body<M>(r, P, K, T, ws, form);
  rin.phase = r.phase;
  rin.rel_par = r.rel_par;
  rin.broken = r.broken;
  return res;
}

template <class M>
__device__ __forceinline__ ClResult cl_pcg_body(ClRun<M>& r, const KParams& P, int K, int T, float* ws, bool form) {
  constexpr int NX = M::NX, NU = M::NU;
  ClResult res{0, false, 0.f, false};
  r.bind(K, T);
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
  res.it = it;
  res.converged = converged && !r.broken;
  return res;
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
