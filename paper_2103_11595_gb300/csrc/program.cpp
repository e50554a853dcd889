// Lowering of a contraction path to a device program (host side).
//
// Each pairwise step C = contract(A, B) over their shared labels is assigned one of three kernel
// classes:
//   GEMM   -- M, N >= 16, K >= 8 and M*N*K >= 2^18: both operands are gathered into real,
//             K-contiguous GEMM operands (the smaller one embedded as [[Re,-Im],[Im,Re]]) and one
//             real GEMM C' = X' Y'^T produces C directly in planar layout with labels
//             (n-bits low, m-bits high). GEMMs run on tcgen05 in the tensor-core precision modes
//             when the shape is tile-aligned, else on CUDA cores.
//   SPLITK -- full contractions to a scalar (the trace) and steps with <= 2^12 outputs and a
//             contracted index of >= 2^10: FP64 partial sums, deterministic final sum.
//   SMALL  -- everything else (gate absorption, outer products, tiny merges): one thread per
//             output element; all SMALL steps of one dependency level share one launch.
// Steps run level by level (level = 1 + the deeper input's level). The arena holds the
// descriptors, the packed inputs, the FP64 result area and a work region whose offsets come from
// a first-fit allocator replaying the launch order, so buffers are reused as soon as their last
// reader has been enqueued.
#include "program.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <stdexcept>

#include "kernels.h"

namespace ajf {
namespace {

constexpr size_t kAlign = 256;
constexpr int64_t kPlanSMsDot = 152;  // SMs of a GB300 (grid sizing of the tiled dot)
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

class FirstFit {
 public:
  size_t alloc(size_t bytes) {
    bytes = align_up(std::max<size_t>(bytes, 1));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first;
        const size_t rest = it->second - bytes;
        free_.erase(it);
        if (rest) free_[off + bytes] = rest;
        return off;
      }
    }
    const size_t off = top_;
    top_ += bytes;
    peak_ = std::max(peak_, top_);
    return off;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(std::max<size_t>(bytes, 1));
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
        it = pv;
      }
    }
    if (it->first + it->second == top_) {
      top_ = it->first;
      free_.erase(it);
    }
  }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;
  size_t top_ = 0, peak_ = 0;
};

BitMap make_map(const std::vector<int>& idx_labels, const std::vector<int>& tensor_labels) {
  BitMap m;
  std::memset(&m, 0, sizeof(m));
  if (idx_labels.size() > static_cast<size_t>(kMaxBits)) throw std::runtime_error("index wider than 48 bits");
  m.nbits = static_cast<int32_t>(idx_labels.size());
  for (size_t i = 0; i < idx_labels.size(); ++i) {
    int pos = -1;
    for (size_t j = 0; j < tensor_labels.size(); ++j)
      if (tensor_labels[j] == idx_labels[i]) { pos = static_cast<int>(j); break; }
    m.pos[i] = static_cast<int8_t>(pos);
  }
  return m;
}

bool contains(const std::vector<int>& v, int x) { return std::find(v.begin(), v.end(), x) != v.end(); }

enum Cls { C_SMALL = 0, C_SPLITK = 1, C_GEMM = 2, C_DOT = 3 };
constexpr int kDotTileBits = 10;

struct StepInfo {
  int cls = C_SMALL;
  int level = 0;
  int a = -1, b = -1;          // input tensor ids (for GEMM: a = X embedded side, b = Y)
  std::vector<int> shared;     // contracted labels (order used for the k index)
  int m = 0, n = 0, k = 0;     // log2 M, N, K
};

int operand_mode(int precision) {
  switch (precision) {
    case AJF_PREC_F64: return OPM_F64;
    case AJF_PREC_F32: return OPM_F32;
    case AJF_PREC_TF32: return OPM_TF32;
    case AJF_PREC_TF32X3: return OPM_TF32X2;
    case AJF_PREC_BF16X3: return OPM_BF16X2;
    case AJF_PREC_F16X3: return OPM_F16X2S;
    default: return OPM_BF16X3;
  }
}
int mode_terms(int mode) {
  return mode == OPM_TF32X2 || mode == OPM_BF16X2 || mode == OPM_F16X2S ? 2 : (mode == OPM_BF16X3 ? 3 : 1);
}
size_t mode_bytes(int mode) { return mode == OPM_F64 ? 8 : (mode >= OPM_BF16X2 ? 2 : 4); }

}  // namespace

Program lower(const Network& net, const Path& path, int precision, size_t inputs_complex, bool tc_ok,
              bool persistent) {
  Program P;
  P.persistent = persistent;
  P.alg = net.alg;
  P.precision = precision;
  // tensors in HBM: complex128 (two FP64 planes), except the products of reduced-precision GEMMs,
  // which are complex64 (two FP32 planes). Such a GEMM promotes every result to one FP32 register
  // sum (or sums its K splits in FP32), and the gathers of the next GEMMs split FP32 values, so
  // nothing is lost; the small steps keep FP64 results, whose rounding would otherwise add up
  // over the hundreds of gate absorptions of a network. Traces, sum |t|^2, F and 1 - F are FP64
  // in every mode.
  P.elem = 8;
  const int L = static_cast<int>(net.leaf_labels.size());
  const int S = static_cast<int>(path.steps.size());
  std::vector<std::vector<int>> labels(L + S);
  std::vector<int> level(L + S, 0);
  for (int i = 0; i < L; ++i) labels[i] = net.leaf_labels[i];
  std::vector<StepInfo> info(S);

  // ---- classify steps and fix every intermediate's label order
  for (int s = 0; s < S; ++s) {
    const PathStep& st = path.steps[s];
    const auto& la = labels[st.a];
    const auto& lb = labels[st.b];
    StepInfo& I = info[s];
    I.level = 1 + std::max(level[st.a], level[st.b]);
    level[L + s] = I.level;
    std::vector<int> fa, fb, sh;
    for (int x : la) (contains(lb, x) ? sh : fa).push_back(x);
    for (int x : lb)
      if (!contains(la, x)) fb.push_back(x);
    const int rc = static_cast<int>(fa.size() + fb.size());
    const int rk = static_cast<int>(sh.size());
    const int ma = static_cast<int>(fa.size()), nb = static_cast<int>(fb.size());
    const double mnk = std::ldexp(1.0, ma + nb + rk);
    std::vector<int> out;
    if (persistent) {
      // one thread block runs the step: a warp per output where the contraction is long and
      // the output short, a thread per output otherwise
      const bool a_big = la.size() >= lb.size();
      I.cls = (rc == 0 || (rc <= 6 && rk >= 8)) ? C_SPLITK : C_SMALL;
      I.a = st.a;
      I.b = st.b;
      I.shared = sh;
      const auto& big = a_big ? fa : fb;
      const auto& small = a_big ? fb : fa;
      out = big;
      out.insert(out.end(), small.begin(), small.end());
    } else if (rc == 0) {
      I.cls = rk >= kDotTileBits ? C_DOT : C_SPLITK;
      I.a = st.a;
      I.b = st.b;
      I.shared = sh;
    } else if (ma >= 4 && nb >= 4 && rk >= 3 && mnk >= std::ldexp(1.0, 18)) {
      I.cls = C_GEMM;
      const bool a_is_x = la.size() <= lb.size();
      const int x = a_is_x ? st.a : st.b, y = a_is_x ? st.b : st.a;
      const auto& lx = labels[x];
      const auto& ly = labels[y];
      std::vector<int> xf, yf, kk;
      for (int v : lx)
        if (!contains(ly, v)) xf.push_back(v);
      for (int v : ly) (contains(lx, v) ? kk : yf).push_back(v);
      I.a = x;
      I.b = y;
      I.shared = kk;  // in Y's bit order
      I.m = static_cast<int>(xf.size());
      I.n = static_cast<int>(yf.size());
      I.k = static_cast<int>(kk.size());
      out = yf;
      out.insert(out.end(), xf.begin(), xf.end());
    } else {
      const bool a_big = la.size() >= lb.size();
      I.cls = (rc <= 12 && rk >= 10) ? C_SPLITK : C_SMALL;
      I.a = st.a;
      I.b = st.b;
      I.shared = sh;
      const auto& big = a_big ? fa : fb;
      const auto& small = a_big ? fb : fa;
      out = big;
      out.insert(out.end(), small.begin(), small.end());
    }
    labels[L + s] = out;
    if (static_cast<int>(out.size()) != static_cast<int>(st.out.size()))
      throw std::runtime_error("internal: step output rank mismatch");
    // (a rough traffic figure: complex128 throughout)
    const double bytes = (std::ldexp(1.0, static_cast<int>(la.size())) + std::ldexp(1.0, static_cast<int>(lb.size())) +
                          std::ldexp(1.0, rc)) * 2.0 * P.elem;
    P.flops += 8.0 * mnk;
    P.bytes += bytes;
    if (I.cls == C_GEMM) {
      P.gemm_flops += 8.0 * mnk;
      P.gemm_bytes += bytes;
      P.n_gemm++;
    }
  }

  // ---- execution order: by level, then class, then path order
  std::vector<int> order(S);
  for (int s = 0; s < S; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    if (info[x].level != info[y].level) return info[x].level < info[y].level;
    return info[x].cls < info[y].cls;
  });
  std::vector<int> exec_pos(S);
  for (int i = 0; i < S; ++i) exec_pos[order[i]] = i;
  std::vector<int> last_use(L + S, -1);
  for (int s = 0; s < S; ++s) {
    last_use[path.steps[s].a] = std::max(last_use[path.steps[s].a], exec_pos[s]);
    last_use[path.steps[s].b] = std::max(last_use[path.steps[s].b], exec_pos[s]);
  }
  std::vector<char> is_final(L + S, 0);
  for (int id : path.final_ids) is_final[id] = 1;

  // ---- arena: work region offsets by first fit in launch order
  FirstFit ff;
  std::vector<size_t> toff(L + S, 0);
  std::vector<char> t32(L + S, 0);  // complex64 tensors: the products of reduced-precision GEMMs
  auto elem = [&](int id) -> size_t { return t32[id] ? 4 : 8; };
  auto tensor_bytes = [&](int id) { return 2 * (size_t(1) << labels[id].size()) * elem(id); };
  for (int i = 0; i < L; ++i) toff[i] = ff.alloc(tensor_bytes(i));
  auto release_dead = [&](int upto_pos, const std::vector<int>& ids) {
    for (int id : ids)
      if (!is_final[id] && last_use[id] <= upto_pos) ff.release(toff[id], tensor_bytes(id));
  };

  const int mode = operand_mode(precision);
  const int terms = mode_terms(mode);
  const size_t eb = mode_bytes(mode);
  // tensor-core operand kind: 0 TF32, 1 bf16, 2 fp16 with per-row-block scales
  const int tc_kind = mode == OPM_F16X2S ? 2 : ((mode >= OPM_BF16X2) ? 1 : 0);
  const bool scaled = mode == OPM_F16X2S;
  int scalar_slots = 0;
  size_t partials = 0;

  // Launch records hold work-region-relative byte offsets; descriptors hold element offsets
  // relative to the work region too. Both are rebased after the layout is known.
  struct PendingGemm {
    int launch;
  };
  std::vector<int> gemm_launches;

  int i = 0;
  while (i < S) {
    const int s0 = order[i];
    const int cls = info[s0].cls, lev = info[s0].level;
    if (cls == C_SMALL || cls == C_SPLITK || cls == C_DOT) {
      int j = i;
      while (j < S && info[order[j]].level == lev && info[order[j]].cls == cls) ++j;
      Launch ln;
      ln.kind = cls == C_SMALL ? LK_SMALL : (cls == C_SPLITK ? LK_SPLITK : LK_DOT);
      ln.op_f64 = precision == AJF_PREC_F64 ? 1 : 0;  // tiled dot: FP32 products in reduced modes
      ln.first = static_cast<int>(P.steps.size());
      ln.count = j - i;
      int blocks = 0;
      size_t smem = 0;
      std::vector<int> consumed;
      for (int t = i; t < j; ++t) {
        const int s = order[t];
        const StepInfo& I = info[s];
        const int c = L + s;
        toff[c] = labels[c].empty() ? 0 : ff.alloc(tensor_bytes(c));
        StepDev d;
        std::memset(&d, 0, sizeof(d));
        const auto& la = labels[I.a];
        const auto& lb = labels[I.b];
        d.a = static_cast<int64_t>(toff[I.a] / elem(I.a));
        d.b = static_cast<int64_t>(toff[I.b] / elem(I.b));
        d.c = static_cast<int64_t>(toff[c] / elem(c));
        d.fa = t32[I.a];
        d.fb = t32[I.b];
        d.pa = int64_t(1) << la.size();
        d.pb = int64_t(1) << lb.size();
        d.pc = int64_t(1) << labels[c].size();
        d.oa = make_map(labels[c], la);
        d.ob = make_map(labels[c], lb);
        // contracted bits ordered by A's positions
        std::vector<int> kl;
        for (int x : la)
          if (contains(lb, x)) kl.push_back(x);
        d.ka = make_map(kl, la);
        d.kb = make_map(kl, lb);
        d.rc = static_cast<int32_t>(labels[c].size());
        d.rk = static_cast<int32_t>(kl.size());
        d.block0 = blocks;
        d.scalar_slot = -1;
        if (cls == C_SMALL) {
          const int64_t nout = int64_t(1) << d.rc;
          blocks += static_cast<int>(std::min<int64_t>((nout + 255) / 256, 8192));
        } else if (cls == C_DOT) {
          // tile bits: the contracted bits on A's five lowest positions, then those on B's five
          // lowest, topped up from A's order (kl follows A's bit order)
          std::vector<int> bits;
          auto add = [&](int i) {
            if (static_cast<int>(bits.size()) < kDotTileBits && !contains(bits, i)) bits.push_back(i);
          };
          std::vector<int> by_b(d.rk);
          for (int q = 0; q < d.rk; ++q) by_b[q] = q;
          std::sort(by_b.begin(), by_b.end(), [&](int x, int y) { return d.kb.pos[x] < d.kb.pos[y]; });
          for (int q = 0; q < 5 && q < d.rk; ++q) add(q);
          for (int q = 0; q < 5 && q < d.rk; ++q) add(by_b[q]);
          for (int q = 0; q < d.rk; ++q) add(q);
          std::vector<int> tla = bits, tlb = bits;
          std::sort(tla.begin(), tla.end(), [&](int x, int y) { return d.ka.pos[x] < d.ka.pos[y]; });
          std::sort(tlb.begin(), tlb.end(), [&](int x, int y) { return d.kb.pos[x] < d.kb.pos[y]; });
          d.ntl = static_cast<int32_t>(bits.size());
          for (int q = 0; q < d.ntl; ++q) {
            d.tl[q] = static_cast<int8_t>(tla[q]);
            d.tlb[q] = static_cast<int8_t>(tlb[q]);
          }
          const int64_t tiles = int64_t(1) << (d.rk - d.ntl);
          // at most 4 blocks per SM (152 SMs): each block amortises its offset-table set-up over
          // more tiles (measured on the mid workload against 8 per SM: 1.88 -> 1.79 ms per step);
          // 3 per SM for the staged FP32 form (three tiles of shared-memory stages per block)
          const int64_t per_sm = dot_staged(d, precision != AJF_PREC_F64) ? 3 : 4;
          const int64_t nsplit = std::max<int64_t>(1, std::min<int64_t>(tiles, per_sm * kPlanSMsDot));
          d.nsplit = static_cast<int32_t>(nsplit);
          d.poff = static_cast<int64_t>(partials);
          partials += static_cast<size_t>(nsplit);
          d.scalar_slot = scalar_slots++;
          blocks += static_cast<int>(nsplit);
        } else {
          const int64_t nout = int64_t(1) << d.rc;
          int64_t nsplit = std::max<int64_t>(1, std::min<int64_t>((int64_t(1) << d.rk) / 2048, 512));
          nsplit = std::max<int64_t>(1, std::min<int64_t>(nsplit, 16384 / nout));
          d.nsplit = static_cast<int32_t>(nsplit);
          d.poff = static_cast<int64_t>(partials);
          partials += static_cast<size_t>(nout * nsplit);
          if (d.rc == 0) d.scalar_slot = scalar_slots++;
          blocks += static_cast<int>(nout * nsplit);
        }
        smem = std::max(smem, cls == C_DOT ? dot_smem_bytes(d, precision != AJF_PREC_F64) : step_table_bytes(d));
        ln.flops += 8.0 * std::ldexp(1.0, d.rc + d.rk);
        ln.bytes += (std::ldexp(1.0, static_cast<int>(la.size())) * elem(I.a) +
                     std::ldexp(1.0, static_cast<int>(lb.size())) * elem(I.b) +
                     (d.rc ? std::ldexp(1.0, d.rc) * elem(c) : 0.0)) * 2.0;
        P.steps.push_back(d);
        consumed.push_back(I.a);
        consumed.push_back(I.b);
      }
      ln.blocks = blocks;
      ln.smem = smem;
      P.launches.push_back(ln);
      release_dead(j - 1, consumed);
      i = j;
    } else {
      const int s = s0;
      const StepInfo& I = info[s];
      const int c = L + s;
      const auto& lx = labels[I.a];
      const auto& ly = labels[I.b];
      std::vector<int> xf, yf;
      for (int v : lx)
        if (!contains(I.shared, v)) xf.push_back(v);
      for (int v : ly)
        if (!contains(I.shared, v)) yf.push_back(v);
      const int64_t Mt = int64_t(1) << (I.m + 1), Nt = int64_t(1) << I.n, Kt = int64_t(1) << (I.k + 1);
      const bool use_tc = tc_ok && precision >= AJF_PREC_TF32 && tc_gemm_supported(Mt, Nt, Kt, tc_kind);
      const bool op_f64 = !use_tc && precision == AJF_PREC_F64;
      const int gmode = use_tc ? mode : (op_f64 ? OPM_F64 : OPM_F32);
      const int gterms = use_tc ? terms : 1;
      const size_t geb = use_tc ? eb : (op_f64 ? 8 : 4);
      const size_t xbytes = size_t(Mt) * size_t(Kt) * geb, ybytes = size_t(Nt) * size_t(Kt) * geb;
      size_t xo[3] = {0, 0, 0}, yo[3] = {0, 0, 0};
      for (int t = 0; t < gterms; ++t) xo[t] = ff.alloc(xbytes);
      for (int t = 0; t < gterms; ++t) yo[t] = ff.alloc(ybytes);
      // scaled fp16 operands: one FP32 power of two per row and 128-byte K block, [K block][row]
      const size_t kblk = use_tc && scaled ? (size_t(Kt) * geb + 127) / 128 : 0;
      const size_t xsb = kblk * size_t(Mt) * 4, ysb = kblk * size_t(Nt) * 4;
      if (kblk) {
        xo[2] = ff.alloc(xsb);
        yo[2] = ff.alloc(ysb);
      }
      // permute launch (X and Y)
      PermDev px, py;
      std::memset(&px, 0, sizeof(px));
      std::memset(&py, 0, sizeof(py));
      px.src = static_cast<int64_t>(toff[I.a] / elem(I.a));
      px.src_f32 = t32[I.a];
      px.plane = int64_t(1) << lx.size();
      px.rows = make_map(xf, lx);
      px.cols = make_map(I.shared, lx);
      px.rbits = I.m;
      px.kbits = I.k;
      px.embed = 1;
      px.rows_fast = contains(xf, lx[0]) ? 1 : 0;
      px.mode = gmode;
      py.src = static_cast<int64_t>(toff[I.b] / elem(I.b));
      py.src_f32 = t32[I.b];
      py.plane = int64_t(1) << ly.size();
      py.rows = make_map(yf, ly);
      py.cols = make_map(I.shared, ly);
      py.rbits = I.n;
      py.kbits = I.k;
      py.embed = 0;
      py.rows_fast = contains(yf, ly[0]) ? 1 : 0;
      py.mode = gmode;
      for (int t = 0; t < 3; ++t) {
        px.dst[t] = static_cast<int64_t>(xo[t]);
        py.dst[t] = static_cast<int64_t>(yo[t]);
      }
      Launch lp;
      lp.kind = LK_PERM;
      lp.op_f64 = gmode == OPM_F64 ? 1 : 0;
      lp.first = static_cast<int>(P.perms.size());
      lp.count = 2;
      // tiles of the larger operand (32 x 32 elements, 32 x 64 in the fixed-point split modes);
      // at most four resident blocks per SM (152 on GB300), each walking several tiles, so that
      // a block's lookup-table set-up is shared by its tiles
      const int tile_bits = gmode == OPM_BF16X3 || gmode == OPM_F16X2S ? 11 : 10;
      const int64_t tiles = std::max<int64_t>(int64_t(1) << std::max(0, I.m + I.k - tile_bits),
                                              int64_t(1) << std::max(0, I.n + I.k - tile_bits));
      lp.blocks = static_cast<int>(std::min<int64_t>(std::max<int64_t>(tiles, 1), 4 * 152));
      lp.smem = std::max(perm_table_bytes(px), perm_table_bytes(py));
      // gather traffic: both complex operands read once, every operand term written once
      lp.bytes = (std::ldexp(1.0, static_cast<int>(lx.size())) * elem(I.a) +
                  std::ldexp(1.0, static_cast<int>(ly.size())) * elem(I.b)) * 2.0 +
                 static_cast<double>(gterms) * static_cast<double>(xbytes + ybytes);
      P.perms.push_back(px);
      P.perms.push_back(py);
      P.launches.push_back(lp);
      release_dead(exec_pos[s], {I.a, I.b});
      t32[c] = op_f64 ? 0 : 1;  // reduced-precision GEMMs write complex64
      toff[c] = ff.alloc(tensor_bytes(c));
      const int ksplit = use_tc ? tc_gemm_splits(Mt, Nt, Kt, tc_kind) : 1;
      const size_t ws_bytes = ksplit > 1 ? size_t(ksplit) * size_t(Mt) * size_t(Nt) * 4 : 0;  // FP32 partials
      const size_t ws = ws_bytes ? ff.alloc(ws_bytes) : 0;
      Launch lg;
      lg.ksplit = ksplit;
      lg.ws_off = static_cast<int64_t>(ws);
      lg.kind = use_tc ? LK_GEMM_TC : LK_GEMM_SIMT;
      lg.op_f64 = op_f64 ? 1 : 0;
      lg.M = Mt;
      lg.N = Nt;
      lg.K = Kt;
      lg.c_off = static_cast<int64_t>(toff[c]);
      lg.tc_kind = tc_kind;
      if (use_tc) {
        // split terms (hi=0, mid=1, lo=2); the kernel forms every product with i + j < terms
        for (int t = 0; t < gterms; ++t) {
          lg.a_off[t] = static_cast<int64_t>(xo[t]);
          lg.b_off[t] = static_cast<int64_t>(yo[t]);
        }
        if (kblk) {  // the scale arrays ride in the third slot of the offsets
          lg.a_off[2] = static_cast<int64_t>(xo[2]);
          lg.b_off[2] = static_cast<int64_t>(yo[2]);
        }
        lg.npass = gterms;
        P.tensor_cores++;
      } else {
        lg.a_off[0] = static_cast<int64_t>(xo[0]);
        lg.b_off[0] = static_cast<int64_t>(yo[0]);
        lg.npass = 1;
      }
      lg.flops = 8.0 * std::ldexp(1.0, I.m + I.n + I.k);
      lg.bytes = (std::ldexp(1.0, static_cast<int>(lx.size())) * elem(I.a) +
                  std::ldexp(1.0, static_cast<int>(ly.size())) * elem(I.b) +
                  std::ldexp(1.0, static_cast<int>(labels[c].size())) * elem(c)) * 2.0;
      gemm_launches.push_back(static_cast<int>(P.launches.size()));
      P.launches.push_back(lg);
      for (int t = 0; t < gterms; ++t) ff.release(xo[t], xbytes);
      for (int t = 0; t < gterms; ++t) ff.release(yo[t], ybytes);
      if (kblk) {
        ff.release(xo[2], xsb);
        ff.release(yo[2], ysb);
      }
      if (ws_bytes) ff.release(ws, ws_bytes);
      ++i;
    }
  }

  // ---- final reduction
  FinalDev& f = P.fin;
  std::memset(&f, 0, sizeof(f));
  f.open_off = -1;
  f.n_qubits = net.n_qubits;
  f.loops = net.loops;
  f.alg = net.alg;
  int open_id = -1;
  for (int id : path.final_ids)
    if (!labels[id].empty()) open_id = id;
  f.open_bits = static_cast<int32_t>(net.open_labels.size());
  if (open_id >= 0) {
    f.open_off = static_cast<int64_t>(toff[open_id] / elem(open_id));
    f.open_f32 = t32[open_id];
    f.open_plane = int64_t(1) << labels[open_id].size();
    f.open_map = make_map(net.open_labels, labels[open_id]);
    if (labels[open_id].size() != net.open_labels.size()) throw std::runtime_error("internal: open tensor rank");
  } else {
    std::memset(&f.open_map, 0, sizeof(f.open_map));
  }
  f.n_scalars = scalar_slots;
  P.n_scalars = scalar_slots;
  P.n_traces = int64_t(1) << f.open_bits;
  P.final_nchunks = (f.open_map.nbits + 7) / 8;
  P.final_blocks = static_cast<int>(std::min<int64_t>((P.n_traces + 255) / 256, 1024));
  f.nblocks = P.final_blocks;

  // ---- arena layout
  size_t off = 0;
  P.off_desc = off;
  P.off_leaves = off;
  off += align_up(sizeof(LeafDev) * std::max<size_t>(1, net.leaf_specs.size()));
  P.off_steps = off;
  off += align_up(sizeof(StepDev) * std::max<size_t>(1, P.steps.size()));
  P.off_perms = off;
  off += align_up(sizeof(PermDev) * std::max<size_t>(1, P.perms.size()));
  P.off_final = off;
  off += align_up(sizeof(FinalDev));
  P.desc_bytes = off - P.off_desc;
  P.off_inputs = off;
  P.input_bytes = inputs_complex * 16;
  off += align_up(std::max<size_t>(P.input_bytes, 16));
  P.off_result = off;
  off += align_up(4 * sizeof(double));
  P.off_status = off;
  off += align_up(16 * sizeof(int32_t));
  P.off_scalars = off;
  off += align_up(sizeof(double) * 2 * std::max(1, scalar_slots));
  P.off_partial = off;
  P.partial_count = partials;
  off += align_up(sizeof(double) * 2 * std::max<size_t>(1, partials));
  P.off_open_partial = off;
  off += align_up(sizeof(double) * P.final_blocks);
  P.off_traces = off;
  off += align_up(sizeof(double) * 2 * static_cast<size_t>(P.n_traces));
  P.off_work = off;
  P.work_bytes = ff.peak();
  P.arena_bytes = off + ff.peak();

  // ---- rebase work-region offsets to the arena
  const int64_t wel = static_cast<int64_t>(P.off_work / P.elem);
  for (int l = 0; l < L; ++l) {
    const LeafSpec& sp = net.leaf_specs[l];
    LeafDev d;
    std::memset(&d, 0, sizeof(d));
    d.off = static_cast<int64_t>(toff[l] / P.elem) + wel;
    d.plane = int64_t(1) << labels[l].size();
    d.src = sp.src;
    d.kind = sp.kind;
    d.a = sp.a;
    d.nk = sp.nk;
    d.kbits = sp.kbits;
    d.bits = static_cast<int32_t>(labels[l].size());
    d.fix_mask = static_cast<uint16_t>(sp.fix_mask);
    d.fix_val = 0;
    P.leaves.push_back(d);
  }
  const int64_t wel32 = static_cast<int64_t>(P.off_work / 4);  // element offsets of complex64 tensors
  for (auto& d : P.steps) {
    d.a += d.fa ? wel32 : wel;
    d.b += d.fb ? wel32 : wel;
    d.c += wel;
  }
  for (auto& p : P.perms) {
    p.src += p.src_f32 ? wel32 : wel;
    for (int t = 0; t < 3; ++t) p.dst[t] += static_cast<int64_t>(P.off_work);
  }
  for (int li : gemm_launches) {
    Launch& g = P.launches[li];
    for (int t = 0; t < 6; ++t) {
      g.a_off[t] += static_cast<int64_t>(P.off_work);
      g.b_off[t] += static_cast<int64_t>(P.off_work);
    }
    g.c_off += static_cast<int64_t>(P.off_work);
    g.ws_off += static_cast<int64_t>(P.off_work);
  }
  if (f.open_off >= 0) f.open_off += f.open_f32 ? wel32 : wel;
  return P;
}

}  // namespace ajf

// ------------------------------------------------------------------ host-side replay check
//
// Every address a kernel of the program can form is a base offset plus a sum of distinct powers
// of two taken from a BitMap, so the largest one is known without running anything. The check
// replays the launches in stream order and tracks, for every buffer written, the last launch that
// reads it, which is what a device memory checker would catch at run time: accesses outside a
// buffer or the arena region it belongs to, buffers that no earlier launch wrote, and launches
// that overwrite a buffer still to be read (or race with their own reads and writes).

namespace ajf {
namespace {

struct Span {
  size_t lo = 0, hi = 0;  // bytes [lo, hi) of the arena
  bool operator==(const Span& o) const { return lo == o.lo && hi == o.hi; }
};
bool overlaps(const Span& x, const Span& y) { return x.lo < y.hi && y.lo < x.hi; }
std::string span_str(const Span& s) { return "[" + std::to_string(s.lo) + ", " + std::to_string(s.hi) + ")"; }

// Add the positions of `m` (those >= 0) to `used`; false if one repeats or is >= limit_bits.
bool add_positions(const BitMap& m, int limit_bits, uint64_t& used) {
  if (m.nbits < 0 || m.nbits > kMaxBits) return false;
  for (int i = 0; i < m.nbits; ++i) {
    const int p = m.pos[i];
    if (p < 0) continue;
    if (p >= limit_bits || ((used >> p) & 1)) return false;
    used |= uint64_t(1) << p;
  }
  return true;
}

int log2_exact(int64_t x) {
  if (x <= 0 || (x & (x - 1))) return -1;
  int b = 0;
  while ((int64_t(1) << b) < x) ++b;
  return b;
}

}  // namespace

std::string check_program(const Program& P) {
  const size_t work_lo = P.off_work, work_hi = P.off_work + P.work_bytes;
  if (P.arena_bytes != work_hi) return "arena size differs from the end of its work region";
  const int64_t inputs_complex = static_cast<int64_t>(P.input_bytes / 16);
  // a tensor's bytes: element offset and plane in units of its own type (complex64: FP32 planes)
  auto tensor = [&](int64_t off_el, int64_t plane, bool f32 = false) {
    const size_t e = f32 ? 4 : 8;
    return Span{static_cast<size_t>(off_el) * e, static_cast<size_t>(off_el + 2 * plane) * e};
  };
  auto in_work = [&](const Span& s) { return s.lo >= work_lo && s.hi <= work_hi && s.lo < s.hi; };

  // launch units: 0 = leaves, 1.. = P.launches, last = the final FP64 pass
  struct Write {
    Span s;
    int unit;
    int last_read;
  };
  std::vector<Write> writes;
  std::vector<std::vector<Span>> unit_reads(P.launches.size() + 2), unit_writes(P.launches.size() + 2);

  // ---- leaves
  for (size_t l = 0; l < P.leaves.size(); ++l) {
    const LeafDev& L = P.leaves[l];
    const std::string who = "leaf " + std::to_string(l);
    if (L.bits < 0 || L.plane != (int64_t(1) << L.bits)) return who + ": plane is not 2^bits";
    const int full_bits = L.bits + __builtin_popcount(L.fix_mask);
    const int op_bits = L.kind == LEAF_KRAUS_OPEN ? 2 * L.a + L.kbits : (L.kind == LEAF_IDENTITY ? 2 : 2 * L.a);
    if (full_bits != op_bits || full_bits > 16 || (L.fix_val & ~L.fix_mask)) return who + ": sliced bits do not fit";
    int64_t need = 0;  // complex input entries read
    const int64_t dim = int64_t(1) << L.a;
    switch (L.kind) {
      case LEAF_GATE: case LEAF_GATE_CONJ: case LEAF_GATE_DAG: case LEAF_GATE_TRANS: need = dim * dim; break;
      case LEAF_KRAUS_OPEN: need = int64_t(L.nk) * dim * dim; break;
      case LEAF_SUPEROP: {
        const int64_t nd = int64_t(1) << (L.a / 2);
        need = int64_t(L.nk) * nd * nd;
        break;
      }
      default: need = 0;
    }
    if (L.src < 0 || L.src + need > inputs_complex) return who + ": reads past the packed inputs";
    const Span s = tensor(L.off, L.plane);
    if (!in_work(s)) return who + ": " + span_str(s) + " is outside the work region";
    unit_writes[0].push_back(s);
  }

  // ---- steps, gathers and GEMMs
  std::vector<char> slot_used(static_cast<size_t>(std::max(1, P.n_scalars)), 0);
  std::vector<Span> partial_spans;
  for (size_t li = 0; li < P.launches.size(); ++li) {
    const Launch& ln = P.launches[li];
    const int u = static_cast<int>(li) + 1;
    const std::string who = "launch " + std::to_string(li);
    auto& R = unit_reads[u];
    auto& W = unit_writes[u];
    if (ln.kind == LK_SMALL || ln.kind == LK_SPLITK || ln.kind == LK_DOT) {
      if (ln.first < 0 || ln.count < 0 || ln.first + ln.count > static_cast<int>(P.steps.size()))
        return who + ": step range";
      for (int k = ln.first; k < ln.first + ln.count; ++k) {
        const StepDev& d = P.steps[k];
        const std::string ws = who + " step " + std::to_string(k);
        const int ba = log2_exact(d.pa), bb = log2_exact(d.pb);
        if (ba < 0 || bb < 0) return ws + ": operand planes are not powers of two";
        if (d.oa.nbits != d.rc || d.ob.nbits != d.rc || d.ka.nbits != d.rk || d.kb.nbits != d.rk)
          return ws + ": map sizes differ from the step's ranks";
        uint64_t ua = 0, ub = 0;
        if (!add_positions(d.oa, ba, ua) || !add_positions(d.ka, ba, ua)) return ws + ": A addresses repeat or overflow";
        if (!add_positions(d.ob, bb, ub) || !add_positions(d.kb, bb, ub)) return ws + ": B addresses repeat or overflow";
        // every operand bit is an output or a contracted bit: otherwise elements would be skipped
        if (ua != (ba == 64 ? ~0ull : (uint64_t(1) << ba) - 1) || ub != (bb == 64 ? ~0ull : (uint64_t(1) << bb) - 1))
          return ws + ": an operand bit is not addressed";
        const Span sa = tensor(d.a, d.pa, d.fa), sb = tensor(d.b, d.pb, d.fb);
        if (!in_work(sa) || !in_work(sb)) return ws + ": an operand lies outside the work region";
        R.push_back(sa);
        R.push_back(sb);
        if (d.scalar_slot >= 0) {
          if (d.scalar_slot >= P.n_scalars || slot_used[d.scalar_slot]) return ws + ": scalar slot reused or out of range";
          slot_used[d.scalar_slot] = 1;
          if (d.rc != 0) return ws + ": a scalar step has output bits";
        } else {
          if (d.pc != (int64_t(1) << d.rc)) return ws + ": output plane is not 2^rc";
          const Span sc = tensor(d.c, d.pc);
          if (!in_work(sc)) return ws + ": output " + span_str(sc) + " lies outside the work region";
          W.push_back(sc);
        }
        if (ln.kind == LK_DOT) {
          if (d.ntl < 0 || d.ntl > 10 || d.ntl > d.rk) return ws + ": dot tile bits";
          uint32_t ta = 0, tb = 0;
          for (int q = 0; q < d.ntl; ++q) {
            if (d.tl[q] < 0 || d.tl[q] >= d.rk || d.tlb[q] < 0 || d.tlb[q] >= d.rk) return ws + ": dot tile bit range";
            ta |= 1u << d.tl[q];
            tb |= 1u << d.tlb[q];
          }
          if (__builtin_popcount(ta) != d.ntl || ta != tb) return ws + ": dot tile bits repeat";
        }
        if (ln.kind == LK_SPLITK || ln.kind == LK_DOT) {
          const int64_t n = (ln.kind == LK_DOT ? 1 : (int64_t(1) << d.rc)) * d.nsplit;
          if (d.nsplit < 1 || d.poff < 0 || d.poff + n > static_cast<int64_t>(P.partial_count))
            return ws + ": partial sums past their region";
          const Span sp{static_cast<size_t>(d.poff), static_cast<size_t>(d.poff + n)};
          for (auto& o : partial_spans)
            if (overlaps(o, sp)) return ws + ": partial sums shared with another step";
          partial_spans.push_back(sp);
        }
      }
    } else if (ln.kind == LK_PERM) {
      if (ln.count != 2 || ln.first < 0 || ln.first + 2 > static_cast<int>(P.perms.size())) return who + ": gather range";
      for (int k = ln.first; k < ln.first + 2; ++k) {
        const PermDev& g = P.perms[k];
        const std::string ws = who + " gather " + std::to_string(k);
        const int bp = log2_exact(g.plane);
        if (bp < 0 || g.rows.nbits != g.rbits || g.cols.nbits != g.kbits) return ws + ": map sizes";
        uint64_t used = 0;
        if (!add_positions(g.rows, bp, used) || !add_positions(g.cols, bp, used))
          return ws + ": source addresses repeat or overflow";
        if (used != (uint64_t(1) << bp) - 1) return ws + ": a source bit is not addressed";
        const Span src = tensor(g.src, g.plane, g.src_f32);
        if (!in_work(src)) return ws + ": source outside the work region";
        R.push_back(src);
        const size_t rows = size_t(1) << (g.rbits + (g.embed ? 1 : 0)), cols = size_t(1) << (g.kbits + 1);
        const size_t bytes = rows * cols * mode_bytes(g.mode);
        for (int t = 0; t < mode_terms(g.mode); ++t) {
          const Span d{static_cast<size_t>(g.dst[t]), static_cast<size_t>(g.dst[t]) + bytes};
          if (!in_work(d)) return ws + ": operand term " + std::to_string(t) + " outside the work region";
          W.push_back(d);
        }
        if (g.mode == OPM_F16X2S) {  // one FP32 scale per row and 128-byte K block
          const size_t sb = rows * ((cols * mode_bytes(g.mode) + 127) / 128) * 4;
          const Span d{static_cast<size_t>(g.dst[2]), static_cast<size_t>(g.dst[2]) + sb};
          if (!in_work(d)) return ws + ": scale array outside the work region";
          W.push_back(d);
        }
      }
    } else if (ln.kind == LK_GEMM_TC || ln.kind == LK_GEMM_SIMT) {
      if (li == 0 || P.launches[li - 1].kind != LK_PERM) return who + ": GEMM without its gather";
      const Launch& lp = P.launches[li - 1];
      const PermDev& px = P.perms[lp.first];
      const PermDev& py = P.perms[lp.first + 1];
      // the GEMM's shape is the gathers': X' = 2M x 2K (embedded), Y' = N x 2K, one K
      if (px.embed != 1 || py.embed != 0 || px.kbits != py.kbits || px.mode != py.mode ||
          ln.M != (int64_t(2) << px.rbits) || ln.N != (int64_t(1) << py.rbits) || ln.K != (int64_t(2) << px.kbits))
        return who + ": GEMM shape differs from its gathers";
      const size_t eb = mode_bytes(px.mode);
      const int terms = ln.kind == LK_GEMM_TC ? ln.npass : 1;
      if (terms < 1 || terms > 3 || terms != mode_terms(px.mode)) return who + ": operand terms";
      if (log2_exact(ln.M) < 0 || log2_exact(ln.N) < 0 || log2_exact(ln.K) < 0) return who + ": GEMM shape";
      for (int t = 0; t < terms; ++t) {
        const Span a{static_cast<size_t>(ln.a_off[t]), static_cast<size_t>(ln.a_off[t]) + size_t(ln.M) * size_t(ln.K) * eb};
        const Span b{static_cast<size_t>(ln.b_off[t]), static_cast<size_t>(ln.b_off[t]) + size_t(ln.N) * size_t(ln.K) * eb};
        if (!in_work(a) || !in_work(b)) return who + ": operand outside the work region";
        R.push_back(a);
        R.push_back(b);
      }
      if (ln.kind == LK_GEMM_TC && px.mode == OPM_F16X2S) {
        const size_t kb = (size_t(ln.K) * eb + 127) / 128;
        const Span a{static_cast<size_t>(ln.a_off[2]), static_cast<size_t>(ln.a_off[2]) + size_t(ln.M) * kb * 4};
        const Span b{static_cast<size_t>(ln.b_off[2]), static_cast<size_t>(ln.b_off[2]) + size_t(ln.N) * kb * 4};
        if (!in_work(a) || !in_work(b)) return who + ": scale array outside the work region";
        R.push_back(a);
        R.push_back(b);
      }
      // the result: complex64 from a reduced-precision GEMM, complex128 from the FP64 one
      const size_t ce = ln.op_f64 ? 8 : 4;
      const Span c{static_cast<size_t>(ln.c_off), static_cast<size_t>(ln.c_off) + size_t(ln.M) * size_t(ln.N) * ce};
      if (!in_work(c)) return who + ": result outside the work region";
      W.push_back(c);
      if (ln.ksplit > 1) {
        const Span w{static_cast<size_t>(ln.ws_off),
                     static_cast<size_t>(ln.ws_off) + size_t(ln.ksplit) * size_t(ln.M) * size_t(ln.N) * 4};
        if (!in_work(w)) return who + ": K-split workspace outside the work region";
        W.push_back(w);  // written by the GEMM and read back by the split sum of the same launch
      }
    } else {
      return who + ": unknown launch kind";
    }
  }

  // ---- final pass
  const int uf = static_cast<int>(P.launches.size()) + 1;
  const FinalDev& f = P.fin;
  if (f.n_scalars != P.n_scalars) return "final pass: scalar count";
  for (int i = 0; i < P.n_scalars; ++i)
    if (!slot_used[i]) return "final pass: scalar slot " + std::to_string(i) + " is never written";
  if (f.open_off >= 0) {
    const int bo = log2_exact(f.open_plane);
    uint64_t used = 0;
    if (bo < 0 || f.open_map.nbits != f.open_bits || bo != f.open_bits || !add_positions(f.open_map, bo, used) ||
        used != (uint64_t(1) << bo) - 1)
      return "final pass: open-tensor addresses";
    const Span so = tensor(f.open_off, f.open_plane, f.open_f32 != 0);
    if (!in_work(so)) return "final pass: open tensor outside the work region";
    unit_reads[uf].push_back(so);
  } else if (f.open_bits != 0) {
    return "final pass: open bits without an open tensor";
  }
  if ((int64_t(1) << f.open_bits) != P.n_traces) return "final pass: trace count";

  // ---- replay: every read finds the most recent exact write before it; no write overlaps a
  // buffer that a later (or the same) launch still reads, nor another write of its launch
  for (int u = 0; u <= uf; ++u) {
    for (const Span& r : unit_reads[u]) {
      int hit = -1;
      for (int w = static_cast<int>(writes.size()) - 1; w >= 0; --w)
        if (writes[w].unit < u && writes[w].s == r) {
          hit = w;
          break;
        }
      if (hit < 0) return "unit " + std::to_string(u) + " reads " + span_str(r) + " that no earlier launch wrote";
      writes[hit].last_read = std::max(writes[hit].last_read, u);
    }
    for (const Span& w : unit_writes[u]) writes.push_back({w, u, -1});
  }
  // last_read is final now; check the hazards
  for (size_t i = 0; i < writes.size(); ++i) {
    const Write& w = writes[i];
    for (const Span& r : unit_reads[w.unit])
      if (overlaps(w.s, r)) return "unit " + std::to_string(w.unit) + " writes " + span_str(w.s) + " over its own input";
    for (size_t j = 0; j < writes.size(); ++j) {
      if (j == i) continue;
      const Write& v = writes[j];
      if (!overlaps(w.s, v.s)) continue;
      if (v.unit == w.unit)
        return "unit " + std::to_string(w.unit) + " writes overlapping buffers " + span_str(w.s) + " and " +
               span_str(v.s);
      if (v.unit < w.unit && v.last_read >= w.unit)
        return "unit " + std::to_string(w.unit) + " overwrites " + span_str(v.s) + " (written by unit " +
               std::to_string(v.unit) + ") before unit " + std::to_string(v.last_read) + " reads it";
    }
  }
  return "";
}

}  // namespace ajf
