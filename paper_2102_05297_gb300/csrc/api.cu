// Host side of libktune: descriptor validation, constraint tabulation, model
// parsing and padding, search state, and the C ABI entry points (ktune.h).
#include <limits.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace ktune {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }

}  // namespace ktune

using namespace ktune;

#define FAIL(code, msg)   \
  do {                    \
    set_error(msg);       \
    return code;          \
  } while (0)

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                    \
      return e_ == cudaErrorMemoryAllocation ? KTUNE_ENOMEM : KTUNE_ECUDA;              \
    }                                                                                   \
  } while (0)

namespace {

// ---- constraint bytecode (host interpreter used to tabulate groups) -------
struct Span {
  int begin, end;  // [begin, end) of the bytecode
};

int op_args(int op) {
  if (op == KTUNE_OP_VAL || op == KTUNE_OP_CONST) return 1;
  if (op == KTUNE_OP_CONST64) return 2;
  return 0;
}

// Structural check; splits the program into groups that start and end with an
// empty stack.
int split_groups(const int32_t *code, int n, int P, std::vector<Span> &spans) {
  int depth = 0, start = 0;
  for (int i = 0; i < n;) {
    const int op = code[i];
    const int na = op_args(op);
    if (op < KTUNE_OP_VAL || op > KTUNE_OP_CONST64) FAIL(KTUNE_EINVAL, "bytecode: unknown opcode");
    if (na > 0 && i + na >= n) FAIL(KTUNE_EINVAL, "bytecode: missing argument");
    if (op == KTUNE_OP_VAL && (code[i + 1] < 0 || code[i + 1] >= P))
      FAIL(KTUNE_EINVAL, "bytecode: VAL parameter out of range");
    if (op == KTUNE_OP_VAL || op == KTUNE_OP_CONST || op == KTUNE_OP_CONST64) {
      ++depth;
    } else if (op == KTUNE_OP_NOT) {
      if (depth < 1) FAIL(KTUNE_EINVAL, "bytecode: stack underflow");
    } else if (op == KTUNE_OP_REQUIRE) {
      if (depth < 1) FAIL(KTUNE_EINVAL, "bytecode: stack underflow");
      --depth;
    } else {
      if (depth < 2) FAIL(KTUNE_EINVAL, "bytecode: stack underflow");
      --depth;
    }
    if (depth > 16) FAIL(KTUNE_EINVAL, "bytecode: stack deeper than 16");
    i += 1 + na;
    if (depth == 0) {
      if (op != KTUNE_OP_REQUIRE) FAIL(KTUNE_EINVAL, "bytecode: value dropped without REQUIRE");
      spans.push_back({start, i});
      start = i;
    }
  }
  if (depth != 0) FAIL(KTUNE_EINVAL, "bytecode: values left on the stack");
  return KTUNE_OK;
}

int64_t tdiv(int64_t a, int64_t b) {
  if (b == 0) return 0;
  if (b == -1) return (int64_t)(0ull - (uint64_t)a);  // wraps like the rest
  return a / b;                                         // C truncates toward zero
}

bool eval_span(const int32_t *code, Span sp, const int64_t *val) {
  int64_t st[17];
  int d = 0;
  bool ok = true;
  for (int i = sp.begin; i < sp.end;) {
    const int op = code[i];
    switch (op) {
      case KTUNE_OP_VAL: st[d++] = val[code[i + 1]]; i += 2; continue;
      case KTUNE_OP_CONST: st[d++] = code[i + 1]; i += 2; continue;
      case KTUNE_OP_CONST64:
        st[d++] = (int64_t)(((uint64_t)(uint32_t)code[i + 2] << 32) | (uint32_t)code[i + 1]);
        i += 3;
        continue;
      case KTUNE_OP_NOT: st[d - 1] = st[d - 1] == 0; ++i; continue;
      case KTUNE_OP_REQUIRE: ok = ok && st[d - 1] != 0; --d; ++i; continue;
      default: break;
    }
    const int64_t b = st[--d], a = st[d - 1];
    const uint64_t ua = (uint64_t)a, ub = (uint64_t)b;
    int64_t r = 0;
    switch (op) {
      case KTUNE_OP_ADD: r = (int64_t)(ua + ub); break;
      case KTUNE_OP_SUB: r = (int64_t)(ua - ub); break;
      case KTUNE_OP_MUL: r = (int64_t)(ua * ub); break;
      case KTUNE_OP_DIV: r = tdiv(a, b); break;
      case KTUNE_OP_MOD: r = b == 0 ? 0 : (int64_t)(ua - (uint64_t)tdiv(a, b) * ub); break;
      case KTUNE_OP_EQ: r = a == b; break;
      case KTUNE_OP_NE: r = a != b; break;
      case KTUNE_OP_LT: r = a < b; break;
      case KTUNE_OP_LE: r = a <= b; break;
      case KTUNE_OP_GT: r = a > b; break;
      case KTUNE_OP_GE: r = a >= b; break;
      case KTUNE_OP_AND: r = (a != 0) && (b != 0); break;
      case KTUNE_OP_OR: r = (a != 0) || (b != 0); break;
    }
    st[d - 1] = r;
    ++i;
  }
  return ok;
}

int build_groups(ktune_space *s, const int32_t *code, int n) {
  std::vector<Span> spans;
  int rc = split_groups(code, n, s->sa.P, spans);
  if (rc) return rc;
  if ((int)spans.size() > kMaxGroups) FAIL(KTUNE_EINVAL, "more than 64 constraint groups");
  for (const Span &sp : spans) {
    bool uses[KTUNE_MAX_PARAMS] = {false};
    for (int i = sp.begin; i < sp.end; i += 1 + op_args(code[i]))
      if (code[i] == KTUNE_OP_VAL) uses[code[i + 1]] = true;
    GroupDev g{};
    int64_t combos = 1;
    for (int j = 0; j < s->sa.P; ++j)
      if (uses[j]) {
        g.param[g.n++] = (uint8_t)j;
        combos *= s->sa.radix[j];
      }
    if (combos > (1 << 20)) FAIL(KTUNE_EINVAL, "constraint group reads too many value combinations");
    int64_t st = 1;
    for (int i = g.n - 1; i >= 0; --i) {
      g.sub_stride[i] = (uint32_t)st;
      st *= s->sa.radix[g.param[i]];
    }
    g.off_words = (uint32_t)s->table.size();
    std::vector<uint32_t> bits((combos + 31) / 32, 0u);
    int64_t val[KTUNE_MAX_PARAMS] = {0};
    for (int64_t c = 0; c < combos; ++c) {
      int64_t rem = c;
      for (int i = g.n - 1; i >= 0; --i) {
        const int j = g.param[i];
        const int d = (int)(rem % s->sa.radix[j]);
        rem /= s->sa.radix[j];
        val[j] = s->values[s->value_off[j] + d];
      }
      if (eval_span(code, sp, val)) bits[c >> 5] |= 1u << (c & 31);
    }
    s->table.insert(s->table.end(), bits.begin(), bits.end());
    s->groups.push_back(g);
  }
  s->sa.n_groups = (int)s->groups.size();
  return KTUNE_OK;
}

// Constrained-index table (see kCiMaxBits): built when the constrained
// parameters' value combinations number at most kCiMaxBits and there is at
// least one constraint; every combination is checked against every group's
// table.
void build_ci(ktune_space *s) {
  if (s->groups.empty()) return;
  uint32_t used = 0;
  for (const GroupDev &g : s->groups)
    for (int i = 0; i < g.n; ++i) used |= 1u << g.param[i];
  int64_t prod = 1;
  for (int j = s->sa.P - 1; j >= 0; --j)
    if ((used >> j) & 1u) {
      s->ci_stride[j] = (uint32_t)prod;
      prod *= s->sa.radix[j];
      if (prod > kCiMaxBits) {
        for (int q = 0; q < KTUNE_MAX_PARAMS; ++q) s->ci_stride[q] = 0;
        return;
      }
    }
  s->ci_table.assign((size_t)((prod + 31) / 32), 0u);
  for (int64_t c = 0; c < prod; ++c) {
    uint64_t p = 0;   // packed digits of a configuration with this constrained combination
    int64_t rem = c;
    for (int j = s->sa.P - 1; j >= 0; --j)
      if ((used >> j) & 1u) {
        p |= (uint64_t)(rem % s->sa.radix[j]) << (4 * j);
        rem /= s->sa.radix[j];
      }
    if (ktune::host_valid(s, p)) s->ci_table[(size_t)(c >> 5)] |= 1u << (c & 31);
  }
}

// Window tables of the one-word layout (see WinDev): groups in program order
// join the current window while the union of their parameters' digit widths
// stays within kWinBits; each window's table holds, for every value of its
// index, the AND of its groups' constraint bits (0 where a field is not a
// digit of its parameter).
void build_windows(ktune_space *s) {
  const int G = (int)s->groups.size();
  std::vector<std::vector<int>> members;   // groups per window
  std::vector<uint32_t> pmask;             // parameters per window (bit mask)
  auto width_of = [&](uint32_t m) {
    int w = 0;
    for (int j = 0; j < s->sa.P; ++j)
      if ((m >> j) & 1u) w += s->width[j];
    return w;
  };
  for (int g = 0; g < G; ++g) {
    const GroupDev &gr = s->groups[g];
    uint32_t m = 0;
    for (int i = 0; i < gr.n; ++i) m |= 1u << gr.param[i];
    if (width_of(m) > kWinBits) {
      s->generic.push_back((uint8_t)g);
      continue;
    }
    if (!members.empty() && width_of(pmask.back() | m) <= kWinBits) {
      members.back().push_back(g);
      pmask.back() |= m;
    } else {
      members.push_back({g});
      pmask.push_back(m);
    }
  }
  for (size_t w = 0; w < members.size(); ++w) {
    WinDev wd{};
    int bits = 0;
    for (int j = 0; j < s->sa.P; ++j)
      if ((pmask[w] >> j) & 1u) {
        wd.pos[wd.n] = s->pos[j];
        wd.mask[wd.n] = (uint8_t)((1u << s->width[j]) - 1u);
        wd.dst[wd.n] = (uint8_t)bits;
        bits += s->width[j];
        ++wd.n;
      }
    const int words = bits >= 5 ? (1 << (bits - 5)) : 1;
    if ((int)s->win.size() == kMaxWin || (int)s->win_table.size() + words > kWinWords) {
      for (int g : members[w]) s->generic.push_back((uint8_t)g);
      continue;
    }
    wd.bits = (uint8_t)bits;
    wd.off = (uint16_t)s->win_table.size();
    std::vector<uint32_t> tab(words, 0u);
    for (uint32_t v = 0; v < (1u << bits); ++v) {
      uint32_t W = 0;   // the word whose window index is v
      for (int i = 0; i < wd.n; ++i)
        W |= ((v >> wd.dst[i]) & wd.mask[i]) << wd.pos[i];
      bool ok = true;
      for (int g : members[w]) {
        const GroupDev &gr = s->groups[g];
        uint32_t sub = 0;
        for (int i = 0; i < gr.n && ok; ++i) {
          const int p = gr.param[i];
          const uint32_t d = (W >> s->pos[p]) & ((1u << s->width[p]) - 1u);
          if ((int)d >= s->sa.radix[p]) ok = false;
          sub += d * gr.sub_stride[i];
        }
        if (ok) ok = (s->table[gr.off_words + (sub >> 5)] >> (sub & 31)) & 1u;
        if (!ok) break;
      }
      if (ok) tab[v >> 5] |= 1u << (v & 31);
    }
    s->win.push_back(wd);
    s->win_table.insert(s->win_table.end(), tab.begin(), tab.end());
  }
}

}  // namespace

namespace ktune {

uint64_t host_pack(const ktune_space *s, int64_t raw) {
  uint64_t p = 0;
  for (int j = s->sa.P - 1; j >= 0; --j) {
    p |= (uint64_t)(raw % s->sa.radix[j]) << (4 * j);
    raw /= s->sa.radix[j];
  }
  return p;
}

bool host_valid(const ktune_space *s, uint64_t p) {
  for (const GroupDev &g : s->groups) {
    uint32_t sub = 0;
    for (int i = 0; i < g.n; ++i) sub += ((p >> (4 * g.param[i])) & 15u) * g.sub_stride[i];
    if (!((s->table[g.off_words + (sub >> 5)] >> (sub & 31)) & 1u)) return false;
  }
  return true;
}

}  // namespace ktune

namespace {

#define TRY(x)          \
  do {                  \
    int rc_ = (x);      \
    if (rc_) return rc_; \
  } while (0)

// host Philox4x32-10 for the initial c_profile draw (same definition as the
// device copy in device_common.cuh)
uint64_t host_philox_u64(uint64_t seed, uint32_t sid, uint32_t step, uint32_t draw, uint32_t dom) {
  uint32_t c[4] = {draw, step, sid, dom};
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = (uint32_t)p1;
    c[2] = n2;
    c[3] = (uint32_t)p0;
  }
  return (uint64_t)c[0] | ((uint64_t)c[1] << 32);
}

uint64_t mulhi64(uint64_t a, uint64_t b) { return (uint64_t)(((unsigned __int128)a * b) >> 64); }

}  // namespace

namespace ktune {

// Section 3.4: bottlenecks (Eqs. global-read, global-write, local,
// inst_fitted, fp32 and its analogues, maxutil, issue, paral) and the
// Delta-PC reaction (memory: -b; instructions: Eq. fp32_reaction; parallelism:
// +b).  Float64, each formula left to right as printed; percentages read as
// pct / 100; ins_util = min(1, ISSUE_U / 50); bottlenecks clamped to [0, 1],
// Deltas to [-1, 1]; absent counters take neutral values (LOC_O and the
// optional instruction classes 0, SM_E = WARP_E = WARP_NP_E = 100, no thread
// count => no parallelism bottleneck); RT + WT = 0 => memory bottlenecks 0;
// ins_fitted = 0 => instruction fractions 0; WARP_E or WARP_NP_E = 0 count as
// 100.  Built with -ffp-contract=off: no fused multiply-add.
void host_expert(const int *roles, int K, const float *cnt, double r, double cores,
                 float *delta32) {
  double v[KTUNE_PC_N_ROLES] = {0};
  bool has[KTUNE_PC_N_ROLES] = {false};
  v[KTUNE_PC_SM_E] = v[KTUNE_PC_WARP_E] = v[KTUNE_PC_WARP_NP_E] = 100.0;
  for (int k = 0; k < K; ++k) {
    const int ro = roles[k];
    if (ro < KTUNE_PC_INERT && !has[ro]) {
      has[ro] = true;
      v[ro] = (double)cnt[k];
    }
  }
  auto clamp01 = [](double x) { return std::min(1.0, std::max(0.0, x)); };
  auto react = [&](double b) { return b <= r ? 0.0 : -((b - r) / (1.0 - r)); };
  double D[KTUNE_PC_N_ROLES] = {0};
  auto mem = [&](int rt, int wt, int u) {
    const double a = v[rt], b = v[wt], util = v[u];
    double br = 0.0, bw = 0.0;
    if (a + b > 0.0) {
      br = clamp01(a / (a + b) * (util / 100.0));
      bw = clamp01(b / (a + b) * (util / 100.0));
    }
    D[rt] = -br;
    D[wt] = -bw;
  };
  mem(KTUNE_PC_DRAM_RT, KTUNE_PC_DRAM_WT, KTUNE_PC_DRAM_U);
  mem(KTUNE_PC_L2_RT, KTUNE_PC_L2_WT, KTUNE_PC_L2_U);
  mem(KTUNE_PC_SHR_LT, KTUNE_PC_SHR_WT, KTUNE_PC_SHR_U);
  D[KTUNE_PC_TEX_RWT] = -clamp01(v[KTUNE_PC_TEX_U] / 100.0);
  D[KTUNE_PC_LOC_O] = -clamp01(v[KTUNE_PC_LOC_O] / 100.0 *
                               std::max(std::max(v[KTUNE_PC_DRAM_U] / 100.0, v[KTUNE_PC_L2_U] / 100.0),
                                        v[KTUNE_PC_TEX_U] / 100.0));
  double we = v[KTUNE_PC_WARP_E], wn = v[KTUNE_PC_WARP_NP_E];
  if (we == 0.0) we = 100.0;
  if (wn == 0.0) wn = 100.0;
  const double ins_fitted = 32.0 * v[KTUNE_PC_INST_EXE] * (100.0 / we) * (100.0 / wn);
  const double issue_u = v[KTUNE_PC_INST_ISSUE_U];
  const double ins_util = std::min(1.0, issue_u / 50.0);
  const int cls[7] = {KTUNE_PC_INST_F32, KTUNE_PC_INST_F64, KTUNE_PC_INST_INT, KTUNE_PC_INST_MISC,
                      KTUNE_PC_INST_LDST, KTUNE_PC_INST_CONT, KTUNE_PC_INST_BCONV};
  double util_max = 0.0;
  for (int c = 0; c < 7; ++c) {
    const double frac = ins_fitted > 0.0 ? v[cls[c]] / ins_fitted : 0.0;
    util_max = c == 0 ? frac : std::max(util_max, frac);
    D[cls[c]] = react(clamp01(frac * ins_util));
  }
  D[KTUNE_PC_INST_ISSUE_U] = react(clamp01(util_max * ((100.0 - issue_u) / 100.0)));
  D[KTUNE_PC_SM_E] = clamp01((100.0 - v[KTUNE_PC_SM_E]) / 100.0);
  if (has[KTUNE_PC_GLOBAL])
    D[KTUNE_PC_GLOBAL] = clamp01(std::max(0.0, (cores * 5.0 - v[KTUNE_PC_GLOBAL]) / (cores * 5.0)));
  bool seen[KTUNE_PC_N_ROLES] = {false};
  for (int k = 0; k < K; ++k) {
    const int ro = roles[k];
    float d = 0.0f;
    if (ro < KTUNE_PC_INERT && !seen[ro]) {
      seen[ro] = true;
      d = (float)std::min(1.0, std::max(-1.0, D[ro]));
    }
    delta32[k] = d;
  }
}

}  // namespace ktune

extern "C" {

int ktune_abi_version(void) { return 100; }

const char *ktune_last_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------------------
int ktune_space_create(const ktune_space_desc *d, int flags, void *stream, ktune_space **out) {
  if (!d || !out) FAIL(KTUNE_EINVAL, "null argument");
  *out = nullptr;
  if (flags != KTUNE_MATERIALISE && flags != KTUNE_ON_THE_FLY) FAIL(KTUNE_EINVAL, "bad flags");
  if (d->n_params < 1 || d->n_params > KTUNE_MAX_PARAMS) FAIL(KTUNE_EINVAL, "n_params out of range");
  if (!d->n_values || !d->values) FAIL(KTUNE_EINVAL, "null value lists");
  if (d->n_bytecode < 0 || (d->n_bytecode > 0 && !d->bytecode)) FAIL(KTUNE_EINVAL, "bad bytecode");
  ktune_space *s = new (std::nothrow) ktune_space();
  if (!s) FAIL(KTUNE_ENOMEM, "host allocation");
  auto cleanup = [&](int rc) {
    ktune_space_destroy(s);
    return rc;
  };
  cudaGetDevice(&s->device);
  s->flags = flags;
  s->sa.P = d->n_params;
  long double raw = 1;
  int off = 0;
  for (int j = 0; j < d->n_params; ++j) {
    const int r = d->n_values[j];
    if (r < 1 || r > KTUNE_MAX_VALUES) {
      set_error("n_values out of range");
      return cleanup(KTUNE_EINVAL);
    }
    s->sa.radix[j] = r;
    s->value_off.push_back(off);
    for (int i = 0; i < r; ++i) {
      if (i && d->values[off + i] <= d->values[off + i - 1]) {
        set_error("value lists must be strictly ascending");
        return cleanup(KTUNE_EINVAL);
      }
      s->values.push_back(d->values[off + i]);
    }
    off += r;
    raw *= r;
  }
  if (raw >= (long double)(1ll << 40)) {
    set_error("raw space size must be below 2^40");
    return cleanup(KTUNE_EINVAL);
  }
  s->sa.n_raw = (int64_t)raw;
  int64_t st = 1;
  for (int j = d->n_params - 1; j >= 0; --j) {
    s->sa.stride[j] = st;
    st *= s->sa.radix[j];
  }
  int rc = build_groups(s, d->bytecode, d->n_bytecode);
  if (rc) return cleanup(rc);
  {  // narrow layout: ceil(log2 radix) bits per digit, parameter 0 lowest
    int bits = 0;
    for (int j = 0; j < d->n_params; ++j) {
      int w = 1;
      while ((1 << w) < s->sa.radix[j]) ++w;
      s->pos[j] = (uint8_t)std::min(bits, 255);
      s->width[j] = (uint8_t)w;
      bits += w;
    }
    s->narrow = bits <= 32;
  }
  if (s->narrow) {
    build_windows(s);
    build_ci(s);
  }

  cudaStream_t cs = (cudaStream_t)stream;
  if ((rc = dalloc(&s->d_groups, s->groups.size()))) return cleanup(rc);
  if ((rc = dalloc(&s->d_table, s->table.size()))) return cleanup(rc);
  if ((rc = dalloc(&s->d_win_table, std::max<size_t>(1, s->win_table.size())))) return cleanup(rc);
  if (!s->ci_table.empty()) {
    if ((rc = dalloc(&s->d_ci_table, s->ci_table.size()))) return cleanup(rc);
    if (cudaMemcpyAsync(s->d_ci_table, s->ci_table.data(), s->ci_table.size() * 4,
                        cudaMemcpyHostToDevice, (cudaStream_t)stream) != cudaSuccess) {
      set_error("descriptor upload failed");
      return cleanup(KTUNE_ECUDA);
    }
  }
  if (!s->win_table.empty() &&
      cudaMemcpyAsync(s->d_win_table, s->win_table.data(), s->win_table.size() * 4,
                      cudaMemcpyHostToDevice, (cudaStream_t)stream) != cudaSuccess) {
    set_error("descriptor upload failed");
    return cleanup(KTUNE_ECUDA);
  }
  if (!s->groups.empty()) {
    if (cudaMemcpyAsync(s->d_groups, s->groups.data(), s->groups.size() * sizeof(GroupDev),
                        cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaMemcpyAsync(s->d_table, s->table.data(), s->table.size() * 4, cudaMemcpyHostToDevice,
                        cs) != cudaSuccess) {
      set_error("descriptor upload failed");
      return cleanup(KTUNE_ECUDA);
    }
  }
  s->n_tiles = (s->sa.n_raw + kEnumTileRaw - 1) / kEnumTileRaw;
  int32_t *d_count = nullptr;
  if ((rc = dalloc(&d_count, s->n_tiles))) return cleanup(rc);
  if ((rc = dalloc(&s->d_tile_offset, s->n_tiles + 1))) {
    cudaFree(d_count);
    return cleanup(rc);
  }
  launch_enum_count(s->sa, s->d_groups, s->d_table, s->n_tiles, d_count, cs);
  launch_scan_tiles(d_count, s->n_tiles, s->d_tile_offset, cs);
  cudaError_t e = cudaMemcpyAsync(&s->n_valid, s->d_tile_offset + s->n_tiles, sizeof(int64_t),
                                  cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  cudaFree(d_count);
  if (e != cudaSuccess) {
    set_error(std::string("enumeration: ") + cudaGetErrorString(e));
    return cleanup(KTUNE_ECUDA);
  }
  if (flags == KTUNE_ON_THE_FLY) {
    s->tile_offset.resize(s->n_tiles + 1);
    if (cudaMemcpy(s->tile_offset.data(), s->d_tile_offset, (s->n_tiles + 1) * 8,
                   cudaMemcpyDeviceToHost) != cudaSuccess) {
      set_error("tile offsets copy failed");
      return cleanup(KTUNE_ECUDA);
    }
    // the tiles that hold a valid configuration: the on-the-fly decode deals
    // them to the warps in turn and never visits the others
    std::vector<int32_t> ne;
    for (int64_t t = 0; t < s->n_tiles; ++t)
      if (s->tile_offset[t + 1] > s->tile_offset[t]) ne.push_back((int32_t)t);
    s->n_ne_tiles = (int64_t)ne.size();
    if (!ne.empty()) {
      if ((rc = dalloc(&s->d_ne_tiles, ne.size()))) return cleanup(rc);
      if (cudaMemcpy(s->d_ne_tiles, ne.data(), ne.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("tile list upload failed");
        return cleanup(KTUNE_ECUDA);
      }
    }
  }
  if (flags == KTUNE_MATERIALISE) {
    if ((rc = dalloc(&s->d_packed, s->n_valid))) return cleanup(rc);
    launch_enum_write(s->sa, s->d_groups, s->d_table, s->n_tiles, s->d_tile_offset, s->d_packed,
                      cs);
    if (s->narrow) {
      if ((rc = dalloc(&s->d_narrow, s->n_valid))) return cleanup(rc);
      PrepArgs lay{};
      for (int j = 0; j < s->sa.P; ++j) lay.pos[j] = s->pos[j];
      launch_narrow_pack(s->d_packed, s->n_valid, lay, s->d_narrow, cs);
    }
    e = cudaStreamSynchronize(cs);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_error(std::string("enumeration: ") + cudaGetErrorString(e));
      return cleanup(KTUNE_ECUDA);
    }
  }
  *out = s;
  return KTUNE_OK;
}

int ktune_space_destroy(ktune_space *s) {
  if (!s) return KTUNE_OK;
  cudaFree(s->d_groups);
  cudaFree(s->d_table);
  cudaFree(s->d_packed);
  cudaFree(s->d_narrow);
  cudaFree(s->d_win_table);
  cudaFree(s->d_ci_table);
  cudaFree(s->d_tile_offset);
  cudaFree(s->d_ne_tiles);
  delete s;
  return KTUNE_OK;
}

int ktune_space_count(const ktune_space *s, int64_t *n_valid, int64_t *n_raw) {
  if (!s) FAIL(KTUNE_EINVAL, "null space");
  if (n_valid) *n_valid = s->n_valid;
  if (n_raw) *n_raw = s->sa.n_raw;
  return KTUNE_OK;
}

int ktune_space_decode(const ktune_space *s, int64_t raw, int64_t *values_out) {
  if (!s || !values_out) FAIL(KTUNE_EINVAL, "null argument");
  if (raw < 0 || raw >= s->sa.n_raw) FAIL(KTUNE_EINVAL, "raw index out of range");
  const uint64_t p = host_pack(s, raw);
  for (int j = 0; j < s->sa.P; ++j) values_out[j] = s->values[s->value_off[j] + ((p >> (4 * j)) & 15u)];
  return KTUNE_OK;
}

int ktune_space_valid_raw(const ktune_space *s, int64_t first, int64_t count, int64_t *out_raw) {
  if (!s || (!out_raw && count)) FAIL(KTUNE_EINVAL, "null argument");
  if (!s->d_packed) FAIL(KTUNE_ESTATE, "space is not materialised");
  if (first < 0 || count < 0 || first + count > s->n_valid) FAIL(KTUNE_EINVAL, "range out of TS");
  std::vector<uint64_t> p((size_t)count);
  if (count) CK(cudaMemcpy(p.data(), s->d_packed + first, count * 8, cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < count; ++i) {
    int64_t raw = 0;
    for (int j = 0; j < s->sa.P; ++j) raw += (int64_t)((p[i] >> (4 * j)) & 15u) * s->sa.stride[j];
    out_raw[i] = raw;
  }
  return KTUNE_OK;
}

int ktune_space_valid_digits(const ktune_space *s, int64_t first, int64_t count, uint8_t *out) {
  if (!s || (!out && count)) FAIL(KTUNE_EINVAL, "null argument");
  if (!s->d_packed) FAIL(KTUNE_ESTATE, "space is not materialised");
  if (first < 0 || count < 0 || first + count > s->n_valid) FAIL(KTUNE_EINVAL, "range out of TS");
  std::vector<uint64_t> p((size_t)count);
  if (count) CK(cudaMemcpy(p.data(), s->d_packed + first, count * 8, cudaMemcpyDeviceToHost));
  const int P = s->sa.P;
  for (int64_t i = 0; i < count; ++i)
    for (int j = 0; j < P; ++j) out[i * P + j] = (uint8_t)((p[i] >> (4 * j)) & 15u);
  return KTUNE_OK;
}

const uint64_t *ktune_space_packed_device(const ktune_space *s) { return s ? s->d_packed : nullptr; }

// ---------------------------------------------------------------------------
// Kind 3, the least-squares model of Section 3.3.1: after the roles, uint32
// n_sub, uint32 T, float coef[n_sub][K][T].  The space fixes the model's
// shape: its two-valued parameters split 2^nb subspaces, its parameters with
// three or more values are the m regressors (T = 1 + 2m + m(m-1)/2), each
// regressor's value v mapped to u = 2 (log2(1 + v) - lo) / (hi - lo) - 1 over
// its value list (float64 here, stored as float32).
// Model blob kind 2: the measured counters of every configuration of TS (the
// exact-counter experiment of Section 4, Table "tab:pc_bias": a table in place
// of a fitted model), uint64 N then float32 [N][K] in TS order.  Stored as
// one column per counter (the cached-prediction layout).
static int load_table(ktune_space *s, const uint8_t *b, size_t bytes, int K, const std::vector<int> &roles,
                      ktune_model **out) {
  if (!s->d_packed) FAIL(KTUNE_ESTATE, "a counter table needs a materialised space");
  uint64_t n = 0;
  if (bytes < 8) FAIL(KTUNE_EMODEL, "blob truncated");
  memcpy(&n, b, 8);
  if ((int64_t)n != s->n_valid) FAIL(KTUNE_EMODEL, "the table's row count differs from the space's TS");
  if (bytes != 8 + n * (size_t)K * 4) FAIL(KTUNE_EMODEL, "table size does not match N x K");
  const float *rows = reinterpret_cast<const float *>(b + 8);
  const int64_t Np = (s->n_valid + 7) / 8 * 8;
  std::vector<float> cols((size_t)K * Np, 0.0f);
  for (int64_t i = 0; i < s->n_valid; ++i)
    for (int c = 0; c < K; ++c) {
      float v;
      memcpy(&v, rows + (size_t)i * K + c, 4);
      if (!isfinite(v)) FAIL(KTUNE_EMODEL, "non-finite counter in the table");
      cols[(size_t)c * Np + i] = v;
    }
  ktune_model *m = new (std::nothrow) ktune_model();
  if (!m) FAIL(KTUNE_ENOMEM, "host allocation");
  m->space = s;
  m->K = K;
  m->D = 0;
  m->kind = 4;
  m->roles = roles;
  m->table_np = Np;
  int rc;
  if ((rc = dalloc(&m->d_table, cols.size()))) {
    delete m;
    return rc;
  }
  if (cudaMemcpy(m->d_table, cols.data(), cols.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(m->d_table);
    delete m;
    FAIL(KTUNE_ECUDA, "table upload failed");
  }
  *out = m;
  return KTUNE_OK;
}

static int load_lsq(ktune_space *s, const uint8_t *b, size_t bytes, int K, const std::vector<int> &roles,
                    ktune_model **out) {
  LsqDev q{};
  q.K = K;
  const int P = s->sa.P;
  std::vector<float> utab((size_t)P * 16, 0.0f);
  for (int j = 0; j < P; ++j) {
    const int r = s->sa.radix[j];
    if (r == 2) {
      q.bmask |= (uint64_t)1 << (4 * j);
      q.bin[q.nb++] = (uint8_t)j;
    }
    if (r < 3) continue;
    q.reg[q.m++] = (uint8_t)j;
    const int64_t *v = s->values.data() + s->value_off[j];
    double lo = INFINITY, hi = -INFINITY;
    std::vector<double> lv(r);
    for (int d = 0; d < r; ++d) {
      if (v[d] <= -1) FAIL(KTUNE_EMODEL, "least-squares regressors need values > -1");
      lv[d] = log2(1.0 + (double)v[d]);
      lo = std::min(lo, lv[d]);
      hi = std::max(hi, lv[d]);
    }
    if (!(hi > lo)) FAIL(KTUNE_EMODEL, "least-squares regressor with equal values");
    for (int d = 0; d < r; ++d) utab[(size_t)j * 16 + d] = (float)(2.0 * (lv[d] - lo) / (hi - lo) - 1.0);
  }
  if (q.nb > kLsqMaxBinary) FAIL(KTUNE_EMODEL, "more than 12 two-valued parameters");
  q.T = 1 + 2 * q.m + q.m * (q.m - 1) / 2;
  uint32_t n_sub, T;
  if (bytes < 8) FAIL(KTUNE_EMODEL, "blob truncated");
  memcpy(&n_sub, b, 4);
  memcpy(&T, b + 4, 4);
  if (n_sub != (1u << q.nb) || T != (uint32_t)q.T)
    FAIL(KTUNE_EMODEL, "least-squares shape does not match the space");
  const size_t n_coef = (size_t)n_sub * K * T;
  if (bytes != 8 + 4 * n_coef) FAIL(KTUNE_EMODEL, bytes < 8 + 4 * n_coef ? "blob truncated" : "trailing bytes in blob");
  std::vector<float> coef(n_coef);
  memcpy(coef.data(), b + 8, 4 * n_coef);
  for (float c : coef)
    if (!isfinite(c)) FAIL(KTUNE_EMODEL, "non-finite coefficient");
  ktune_model *m = new (std::nothrow) ktune_model();
  if (!m) FAIL(KTUNE_ENOMEM, "host allocation");
  m->space = s;
  m->K = K;
  m->D = 0;
  m->kind = 3;
  m->roles = roles;
  m->lsq_m = q.m;
  m->lsq_nb = q.nb;
  int rc;
  if ((rc = dalloc(&m->d_lsq, 1)) || (rc = dalloc(&m->d_lsq_utab, utab.size())) ||
      (rc = dalloc(&m->d_lsq_coef, n_coef))) {
    ktune_model_destroy(m);
    return rc;
  }
  q.utab = m->d_lsq_utab;
  q.coef = m->d_lsq_coef;
  if (cudaMemcpy(m->d_lsq_utab, utab.data(), utab.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->d_lsq_coef, coef.data(), n_coef * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->d_lsq, &q, sizeof(q), cudaMemcpyHostToDevice) != cudaSuccess) {
    ktune_model_destroy(m);
    FAIL(KTUNE_ECUDA, "model upload failed");
  }
  *out = m;
  return KTUNE_OK;
}

int ktune_model_load(ktune_space *s, const void *blob, size_t bytes, ktune_model **out) {
  if (!s || !blob || !out) FAIL(KTUNE_EINVAL, "null argument");
  *out = nullptr;
  const uint8_t *b = (const uint8_t *)blob;
  size_t pos = 0;
  auto rd32 = [&](uint32_t *v) {
    if (pos + 4 > bytes) return false;
    memcpy(v, b + pos, 4);
    pos += 4;
    return true;
  };
  uint32_t magic, ver, kind, K;
  if (!rd32(&magic) || !rd32(&ver) || !rd32(&kind) || !rd32(&K)) FAIL(KTUNE_EMODEL, "blob truncated");
  if (magic != 0x314D544Bu || ver != 1) FAIL(KTUNE_EMODEL, "bad magic or version");
  if (kind != 1 && kind != 2 && kind != 3) FAIL(KTUNE_EMODEL, "unsupported model kind");
  if (K < 1 || K > KTUNE_MAX_COUNTERS) FAIL(KTUNE_EMODEL, "K out of range");
  std::vector<int> roles(K);
  for (uint32_t k = 0; k < K; ++k) {
    uint32_t r;
    if (!rd32(&r)) FAIL(KTUNE_EMODEL, "blob truncated");
    if ((int)r < 0 || (int)r >= KTUNE_PC_N_ROLES) FAIL(KTUNE_EMODEL, "bad counter role");
    roles[k] = (int)r;
  }
  if (kind == 3) return load_lsq(s, b + pos, bytes - pos, (int)K, roles, out);
  if (kind == 2) return load_table(s, b + pos, bytes - pos, (int)K, roles, out);
  struct Tree {
    std::vector<int32_t> f, t, l, r;
    std::vector<float> v;
  };
  std::vector<Tree> trees(K);
  int D = 1;
  for (uint32_t k = 0; k < K; ++k) {
    uint32_t n;
    if (!rd32(&n) || n < 1 || n > (1u << (KTUNE_MAX_DEPTH + 1))) FAIL(KTUNE_EMODEL, "bad node count");
    if (pos + (size_t)n * 20 > bytes) FAIL(KTUNE_EMODEL, "blob truncated");
    Tree &T = trees[k];
    T.f.resize(n); T.t.resize(n); T.l.resize(n); T.r.resize(n); T.v.resize(n);
    memcpy(T.f.data(), b + pos, 4 * n); pos += 4 * n;
    memcpy(T.t.data(), b + pos, 4 * n); pos += 4 * n;
    memcpy(T.l.data(), b + pos, 4 * n); pos += 4 * n;
    memcpy(T.r.data(), b + pos, 4 * n); pos += 4 * n;
    memcpy(T.v.data(), b + pos, 4 * n); pos += 4 * n;
    // every node reached exactly once from the root, depth bounded
    std::vector<int> depth(n, -1);
    std::vector<int> stack{0};
    depth[0] = 0;
    size_t seen = 0;
    while (!stack.empty()) {
      const int i = stack.back();
      stack.pop_back();
      ++seen;
      if (depth[i] > KTUNE_MAX_DEPTH) FAIL(KTUNE_EMODEL, "tree deeper than KTUNE_MAX_DEPTH");
      if (T.f[i] < 0) {
        if (!isfinite(T.v[i])) FAIL(KTUNE_EMODEL, "non-finite leaf value");
        D = std::max(D, depth[i]);
        continue;
      }
      if (T.f[i] >= s->sa.P) FAIL(KTUNE_EMODEL, "tree feature beyond the space's parameters");
      if (T.t[i] < 0) FAIL(KTUNE_EMODEL, "negative threshold");
      for (int c : {T.l[i], T.r[i]}) {
        if (c < 1 || c >= (int)n || depth[c] != -1) FAIL(KTUNE_EMODEL, "bad child index");
        depth[c] = depth[i] + 1;
        stack.push_back(c);
      }
    }
    (void)seen;
  }
  if (pos != bytes) FAIL(KTUNE_EMODEL, "trailing bytes in blob");
  // pad into complete trees of depth D
  const int L = 1 << D;
  std::vector<uint8_t> nodes((size_t)K * L, 0);
  std::vector<float> leaves((size_t)K * L, 0.0f);
  for (uint32_t k = 0; k < K; ++k) {
    const Tree &T = trees[k];
    uint8_t *nd = nodes.data() + (size_t)k * L;
    float *lv = leaves.data() + (size_t)k * L;
    // (source node, padded position, level)
    std::vector<std::array<int, 3>> st{{0, 0, 0}};
    while (!st.empty()) {
      auto [i, pos_, lev] = st.back();
      st.pop_back();
      if (lev == D) {
        lv[pos_ - (L - 1)] = T.v[i];
        continue;
      }
      if (T.f[i] < 0) {
        nd[pos_] = 0x0F;  // feature 0, threshold 15: always left
        st.push_back({i, 2 * pos_ + 1, lev + 1});
        st.push_back({i, 2 * pos_ + 2, lev + 1});  // unreachable copy keeps the table full
        continue;
      }
      const int thr = std::min(T.t[i], 15);
      nd[pos_] = (uint8_t)((T.f[i] << 4) | thr);
      st.push_back({T.l[i], 2 * pos_ + 1, lev + 1});
      st.push_back({T.r[i], 2 * pos_ + 2, lev + 1});
    }
  }
  ktune_model *m = new (std::nothrow) ktune_model();
  if (!m) FAIL(KTUNE_ENOMEM, "host allocation");
  m->space = s;
  m->K = (int)K;
  m->D = D;
  m->roles = roles;
  int rc;
  if ((rc = dalloc(&m->d_nodes, nodes.size())) || (rc = dalloc(&m->d_leaves, leaves.size()))) {
    ktune_model_destroy(m);
    return rc;
  }
  if (cudaMemcpy(m->d_nodes, nodes.data(), nodes.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->d_leaves, leaves.data(), leaves.size() * 4, cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    ktune_model_destroy(m);
    FAIL(KTUNE_ECUDA, "model upload failed");
  }
  *out = m;
  return KTUNE_OK;
}

int ktune_model_destroy(ktune_model *m) {
  if (!m) return KTUNE_OK;
  if (m->kind == 2) {   // the MLP is the caller's
    delete m;
    return KTUNE_OK;
  }
  cudaFree(m->d_nodes);
  cudaFree(m->d_leaves);
  cudaFree(m->d_table);
  cudaFree(m->d_lsq);
  cudaFree(m->d_lsq_utab);
  cudaFree(m->d_lsq_coef);
  delete m;
  return KTUNE_OK;
}

int ktune_model_info(const ktune_model *m, int *K, int *depth) {
  if (!m) FAIL(KTUNE_EINVAL, "null model");
  if (K) *K = m->K;
  if (depth) *depth = m->D;
  return KTUNE_OK;
}

int ktune_model_predict_device(const ktune_model *m, int64_t first, int64_t count, float *out,
                               void *stream) {
  if (!m || (!out && count)) FAIL(KTUNE_EINVAL, "null argument");
  const ktune_space *s = m->space;
  if (!s->d_packed) FAIL(KTUNE_ESTATE, "space is not materialised");
  if (first < 0 || count < 0 || first + count > s->n_valid) FAIL(KTUNE_EINVAL, "range out of TS");
  if (m->kind == 2) return ktune_mlp_predict_device(m->mlp, first, count, out, stream);
  if (m->kind == 4) {
    launch_cols_to_rows(m->d_table, m->table_np, m->K, first, count, out, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return KTUNE_OK;
  }
  if (m->kind == 3) {
    launch_lsq_predict(m->d_lsq, s->d_packed + first, count, out, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return KTUNE_OK;
  }
  launch_predict_full(s->d_packed + first, count, m->d_nodes, m->d_leaves, m->K, m->D, out,
                      (cudaStream_t)stream);
  CK(cudaGetLastError());
  return KTUNE_OK;
}

// ---------------------------------------------------------------------------
int ktune_search_create(ktune_space *s, ktune_model *m, const ktune_search_opts *o, void *stream,
                        ktune_search **out) {
  if (!s || !m || !o || !out) FAIL(KTUNE_EINVAL, "null argument");
  *out = nullptr;
  if (m->space != s) FAIL(KTUNE_EINVAL, "model belongs to another space");
  if (o->k < 1 || o->k > KTUNE_MAX_K) FAIL(KTUNE_EINVAL, "k out of range");
  if (o->select != KTUNE_SELECT_SAMPLE && o->select != KTUNE_SELECT_TOPK)
    FAIL(KTUNE_EINVAL, "bad select mode");
  if (!(o->inst_reaction >= 0.0 && o->inst_reaction < 1.0)) FAIL(KTUNE_EINVAL, "inst_reaction not in [0,1)");
  if (!(o->cores > 0.0) || !isfinite(o->gamma)) FAIL(KTUNE_EINVAL, "bad cores or gamma");
  if (s->n_valid == 0) FAIL(KTUNE_EXHAUSTED, "empty tuning space");
  if (m->kind == 2 && (!s->d_packed || o->select != KTUNE_SELECT_SAMPLE))
    FAIL(KTUNE_ESTATE, "MLP models need a materialised space and KTUNE_SELECT_SAMPLE");
  if (m->kind == 4 && o->select != KTUNE_SELECT_SAMPLE)
    FAIL(KTUNE_ESTATE, "counter-table models need KTUNE_SELECT_SAMPLE");
  if (m->kind == 3 && (!s->d_packed || o->select != KTUNE_SELECT_SAMPLE))
    FAIL(KTUNE_ESTATE, "least-squares models need a materialised space and KTUNE_SELECT_SAMPLE");
  const bool otf = s->flags == KTUNE_ON_THE_FLY;
  if (otf && !s->narrow)
    FAIL(KTUNE_ESTATE, "on-the-fly spaces need all digits in one 32-bit word (sum of ceil(log2 n_values) <= 32)");
  if (otf && s->sa.n_raw >= (int64_t)1 << 32) FAIL(KTUNE_EINVAL, "on-the-fly spaces need fewer than 2^32 raw configurations");
  const int64_t N = s->n_valid;
  if (N >= ((int64_t)1 << 32) - 1) FAIL(KTUNE_EINVAL, "more than 2^32 - 2 valid configurations");
  const int64_t n_sub = (N + kSubTile - 1) / kSubTile;
  if ((n_sub + kSuper - 1) / kSuper > kMaxSuper) FAIL(KTUNE_EINVAL, "space too large for the select hierarchy");
  ktune_search *h = new (std::nothrow) ktune_search();
  if (!h) FAIL(KTUNE_ENOMEM, "host allocation");
  h->space = s;
  h->model = m;
  h->opts = *o;
  h->stream = (cudaStream_t)stream;
  h->mode = otf ? 2 : (s->narrow ? 0 : 1);
  h->n_sub = n_sub;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
  // work items: one contiguous range per SM
  std::vector<ItemDev> items;
  {
    const int64_t units = otf ? s->n_tiles : N;
    const int64_t G = std::max<int64_t>(1, std::min<int64_t>(h->num_sms, otf ? units : (units + 4095) / 4096));
    for (int64_t b = 0; b < G; ++b) {
      ItemDev it{};
      it.search = 0;
      it.lo = units * b / G;
      it.hi = units * (b + 1) / G;
      if (it.hi > it.lo) items.push_back(it);
    }
  }
  h->n_items = (int)items.size();
  h->grid = h->n_items;
  size_t tree_bytes = (size_t)pack_tree_bytes(m->D, h->mode != 1);
  if (m->kind == 3)   // the step's coefficient pack, per counter slot
    tree_bytes = std::max<size_t>(16, (size_t)lsq_pack_bytes(m->lsq_m, m->lsq_nb, m->K) / m->K + 16);
  int rc;
  auto fail = [&](int code) {
    ktune_search_destroy(h);
    return code;
  };
  if ((rc = dalloc(&h->d_eval, (N + 31) / 32)) || (rc = dalloc(&h->d_counters, m->K)) ||
      (rc = dalloc(&h->d_pcprof, m->K)) || (rc = dalloc(&h->d_delta, m->K)) ||
      (rc = dalloc(&h->d_nactive, 1)) || (rc = dalloc(&h->d_pack, tree_bytes * m->K)) ||
      (rc = dalloc(&h->d_s, N)) || (rc = dalloc(&h->d_w, N)) || (rc = dalloc(&h->d_subsum, n_sub)) ||
      (rc = dalloc(&h->d_supsum, (n_sub + kSuper - 1) / kSuper)) ||
      (rc = dalloc(&h->d_cand_key, (size_t)h->n_items * KTUNE_MAX_K)) ||
      (rc = dalloc(&h->d_cand_raw, (size_t)h->n_items * KTUNE_MAX_K)) || (rc = dalloc(&h->d_mm, 2)) ||
      (rc = dalloc(&h->d_srch, 1)) || (rc = dalloc(&h->d_steps, 1)) ||
      (rc = dalloc(&h->d_items, h->n_items)) || (rc = dalloc(&h->d_sub_search, n_sub)) ||
      (rc = dalloc(&h->d_out_raw, KTUNE_MAX_K)) || (rc = dalloc(&h->d_out_score, KTUNE_MAX_K)) ||
      (rc = dalloc(&h->d_out_packed, KTUNE_MAX_K)) || (rc = dalloc(&h->d_nout, 1)))
    return fail(rc);
  if (cudaMallocHost((void **)&h->h_counters, KTUNE_MAX_COUNTERS * 4) != cudaSuccess ||
      cudaHostAlloc((void **)&h->hout, sizeof(HostOut), cudaHostAllocMapped) != cudaSuccess ||
      cudaMallocHost((void **)&h->h_nout, 8) != cudaSuccess) {
    set_error("pinned host allocation failed");
    return fail(KTUNE_ENOMEM);
  }
  if (cudaHostGetDevicePointer((void **)&h->hout_dev, h->hout, 0) != cudaSuccess) {
    set_error("mapped host memory is not addressable by the device");
    return fail(KTUNE_ECUDA);
  }
  memset(h->hout, 0, sizeof(HostOut));
  SearchDev &sd = h->sdh;
  sd.packed = s->d_packed;
  sd.narrow = s->d_narrow;
  sd.tile_offset = s->d_tile_offset;
  sd.ne_tiles = s->d_ne_tiles;
  sd.n_ne_tiles = s->n_ne_tiles;
  sd.groups = s->d_groups;
  sd.table = s->d_table;
  sd.N = N;
  sd.mode = h->mode;
  sd.select = o->select;
  sd.sa = s->sa;
  for (int j = 0; j < KTUNE_MAX_PARAMS; ++j) {
    sd.pos[j] = s->pos[j];
    sd.width[j] = s->width[j];
  }
  sd.ci_table = s->d_ci_table;
  sd.ci_words = (int)s->ci_table.size();
  for (int j = 0; j < KTUNE_MAX_PARAMS; ++j) sd.ci_stride[j] = s->ci_stride[j];
  sd.win_table = s->d_win_table;
  sd.n_win = (int)s->win.size();
  sd.win_words = (int)s->win_table.size();
  for (int w = 0; w < sd.n_win; ++w) sd.win[w] = s->win[w];
  sd.n_generic = (int)s->generic.size();
  for (int g = 0; g < sd.n_generic; ++g) sd.generic[g] = s->generic[g];
  {
    int64_t rem = 128;
    for (int j = s->sa.P - 1; j >= 0; --j) {
      sd.inc128[j] = (uint8_t)(rem % s->sa.radix[j]);
      rem /= s->sa.radix[j];
    }
  }
  sd.nodes = m->d_nodes;
  sd.kind = m->kind;
  sd.lsq = m->d_lsq;
  sd.lsq_pack = m->kind == 3;
  sd.leaves = m->d_leaves;
  sd.K = m->K;
  sd.D = m->D;
  for (int i = 0; i < m->K; ++i) sd.roles[i] = (uint8_t)m->roles[i];
  sd.inst_reaction = o->inst_reaction;
  sd.cores = o->cores;
  sd.gamma = o->gamma;
  sd.search_id = o->search_id;
  sd.seed = o->seed;
  sd.eval = h->d_eval;
  sd.pack = h->d_pack;
  sd.pcprof = h->d_pcprof;
  sd.delta = h->d_delta;
  sd.n_active = h->d_nactive;
  sd.mm = h->d_mm;
  sd.s = h->d_s;
  sd.w = h->d_w;
  sd.sub_sum = h->d_subsum;
  sd.super_sum = h->d_supsum;
  sd.cand_key = h->d_cand_key;
  sd.cand_raw = h->d_cand_raw;
  sd.item_begin = 0;
  sd.item_end = h->n_items;
  sd.sub_begin = 0;
  cudaStream_t cs = h->stream;
  if (cudaMemcpyAsync(h->d_srch, &sd, sizeof(sd), cudaMemcpyHostToDevice, cs) != cudaSuccess ||
      cudaMemcpyAsync(h->d_items, items.data(), items.size() * sizeof(ItemDev),
                      cudaMemcpyHostToDevice, cs) != cudaSuccess ||
      cudaMemsetAsync(h->d_sub_search, 0, n_sub * sizeof(int), cs) != cudaSuccess ||
      cudaMemsetAsync(h->d_eval, 0, ((N + 31) / 32) * 4, cs) != cudaSuccess) {
    set_error("search set-up upload failed");
    return fail(KTUNE_ECUDA);
  }
  // initial c_profile: TS[floor(u N / 2^64)], u from Philox domain 1
  const int64_t o0 = (int64_t)mulhi64(host_philox_u64(o->seed, o->search_id, 0, 0, 1), (uint64_t)N);
  int64_t raw = -1;
  if (!otf) {
    uint64_t p = 0;
    if (cudaMemcpyAsync(&p, s->d_packed + o0, 8, cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
        cudaStreamSynchronize(cs) != cudaSuccess) {
      set_error("copy failed");
      return fail(KTUNE_ECUDA);
    }
    raw = 0;
    for (int j = 0; j < s->sa.P; ++j) raw += (int64_t)((p >> (4 * j)) & 15u) * s->sa.stride[j];
  } else {
    const std::vector<int64_t> &to = s->tile_offset;
    const int64_t t = (int64_t)(std::upper_bound(to.begin(), to.end(), o0) - to.begin()) - 1;
    int64_t rank = o0 - to[t];
    for (int64_t r = t * kEnumTileRaw; r < std::min<int64_t>(s->sa.n_raw, (t + 1) * kEnumTileRaw); ++r)
      if (host_valid(s, host_pack(s, r)) && rank-- == 0) {
        raw = r;
        break;
      }
  }
  launch_mark(h->d_eval, o0, cs);
  if (raw < 0 || cudaStreamSynchronize(cs) != cudaSuccess) {
    set_error("search set-up failed");
    return fail(KTUNE_ECUDA);
  }
  h->cprof_raw = raw;
  h->cprof_packed = host_pack(s, raw);
  h->n_evaluated = 1;
  const bool fotf = h->mode == 2 && fused_blocks_per_sm_otf() >= 1;
  const int fshape = fotf ? 2 : fused_blocks_per_sm(1) >= 1 ? 2 : fused_blocks_per_sm(0) >= 1 ? 1 : 0;
  if (m->kind == 1 && (h->mode == 0 || fotf) && fshape) {
    // the whole step as one persistent kernel (the default where it applies)
    const int L = 1 << m->D;
    h->fused_grid = h->num_sms;
    PrepArgs lay{};
    for (int j = 0; j < s->sa.P; ++j) {
      lay.pos[j] = s->pos[j];
      lay.width[j] = s->width[j];
      lay.radix[j] = (uint8_t)s->sa.radix[j];
    }
    const int mm0[2] = {INT_MAX, INT_MIN};
    if ((rc = dalloc(&h->d_fz_words, (size_t)m->K * L)) || (rc = dalloc(&h->d_fz_terms, (size_t)m->K * L)) ||
        (rc = dalloc(&h->d_fz_mm, 2)) || (rc = dalloc(&h->d_fz_phase, 8)) ||
        (rc = dalloc(&h->d_fz_sync, 2)) || (rc = dalloc(&h->d_fz_status, 1)) ||
        (rc = dalloc(&h->d_fz_cand, (size_t)h->fused_grid * KTUNE_MAX_K)) ||
        (fotf && (rc = dalloc(&h->d_fz_list, (size_t)N))))
      return fail(rc);
    if (launch_fused_words(m->d_nodes, m->K, m->D, lay, h->d_fz_words, cs) != cudaSuccess ||
        cudaMemcpyAsync(h->d_fz_mm, mm0, 8, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaMemsetAsync(h->d_fz_sync, 0, 16, cs) != cudaSuccess ||
        cudaMemsetAsync(h->d_fz_status, 0, 4, cs) != cudaSuccess ||
        cudaStreamSynchronize(cs) != cudaSuccess) {
      set_error("fused-step set-up failed");
      return fail(KTUNE_ECUDA);
    }
    // below kFusedDefaultMin configurations the four kernels' lower fixed cost
    // wins (a CUDA graph on a non-default stream: 40 us per step on the
    // 1,824-configuration space, against 46 us for the cooperative launch)
    h->fused = N >= kFusedDefaultMin ? fshape : 0;
  }
  *out = h;
  return KTUNE_OK;
}

static void drop_graph(ktune_search *h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->gexec = nullptr;
  h->graph = nullptr;
  h->prep_node = nullptr;
}

int ktune_search_destroy(ktune_search *h) {
  if (!h) return KTUNE_OK;
  cudaFree(h->d_nbr);
  cudaFree(h->d_nbr_buf);
  cudaFree(h->d_cache);
  cudaFree(h->d_leaf_cache);
  void *fz[] = {h->d_fz_list, h->d_fz_words, h->d_fz_terms, h->d_fz_phase, h->d_fz_mm, h->d_fz_sync, h->d_fz_status, h->d_fz_cand};
  for (void *p : fz) cudaFree(p);
  void *dev[] = {h->d_eval, h->d_counters, h->d_pcprof, h->d_delta, h->d_nactive, h->d_pack,
                 h->d_s, h->d_w, h->d_subsum, h->d_supsum, h->d_cand_key, h->d_cand_raw, h->d_mm, h->d_srch,
                 h->d_steps, h->d_items, h->d_sub_search, h->d_out_raw, h->d_out_score,
                 h->d_out_packed, h->d_nout};
  for (void *p : dev) cudaFree(p);
  void *pin[] = {h->h_counters, h->hout, h->h_nout};
  for (void *p : pin) cudaFreeHost(p);
  for (auto &e : h->ev)
    if (e) cudaEventDestroy(e);
  drop_graph(h);
  delete h;
  return KTUNE_OK;
}

int ktune_search_current(const ktune_search *h, int64_t *raw) {
  if (!h || !raw) FAIL(KTUNE_EINVAL, "null argument");
  *raw = h->cprof_raw;
  return KTUNE_OK;
}

int ktune_search_set_profile(ktune_search *h, int64_t raw) {
  if (!h) FAIL(KTUNE_EINVAL, "null search");
  const ktune_space *s = h->space;
  if (raw < 0 || raw >= s->sa.n_raw) FAIL(KTUNE_EINVAL, "raw index out of range");
  const uint64_t p = host_pack(s, raw);
  if (!host_valid(s, p)) FAIL(KTUNE_EINVAL, "configuration is not valid");
  h->cprof_raw = raw;
  h->cprof_packed = p;
  return KTUNE_OK;
}

int ktune_search_evaluated(const ktune_search *h, int64_t *n) {
  if (!h || !n) FAIL(KTUNE_EINVAL, "null argument");
  *n = h->n_evaluated;
  return KTUNE_OK;
}

// The kernels of one step, in order (recorded into a graph or launched).
static void launch_step_kernels(ktune_search *h, const StepBatch<1> &sb, cudaStream_t st,
                                bool capturing) {
  const ktune_model *m = h->model;
  // while capturing, external records become event nodes of the graph
  auto mark = [&](int i) {
    if (!h->timing) return;
    if (capturing) cudaEventRecordWithFlags(h->ev[i], st, cudaEventRecordExternal);
    else cudaEventRecord(h->ev[i], st);
  };
  mark(0);
  if (h->nbr_radius) {
    // the neighbourhood of c_profile only: score, then select (its own kernels)
    launch_nbr_step(h->d_srch, h->d_steps, sb, h->nbr_C, h->num_sms, st);
    mark(1);
    mark(2);
    mark(3);
    mark(4);
    return;
  }
  if (m->kind == 4) {
    // a measured counter table: the step's set-up with c_profile's row, then
    // Eq. score from the table's columns of the active counters
    launch_table_prep(h->d_srch, h->d_steps, sb, m->d_table, m->table_np, st);
    mark(1);
    launch_cscore(h->d_srch, m->d_table, m->table_np, h->num_sms, st);
  } else if (h->cached) {
    // cached predictions: the step's set-up and c_profile prediction, then
    // Eq. score from the cached columns of the active counters
    if (m->kind == 2) {
      launch_mlp_prep(h->d_srch, h->d_steps, sb, st);
      launch_mlp_fwd(0, m->mlp->dev(), &h->d_steps[0].cprof_packed, 1, h->d_pcprof, nullptr,
                     nullptr, nullptr, nullptr, m->mlp->d_status, 1, st);
      mark(1);
      launch_cscore(h->d_srch, h->d_cache, h->cache_np, h->num_sms, st);
    } else if (m->kind == 3) {
      launch_lsq_prep(h->d_srch, h->d_steps, sb, 0, st);
      mark(1);
      launch_cscore(h->d_srch, h->d_cache, h->cache_np, h->num_sms, st);
    } else {
      launch_bprep(h->d_srch, h->d_steps, sb, 1, m->K, m->D, st);
      mark(1);
      const bool narrow = h->mode != 1;
      const int L = 1 << m->D;
      launch_cscore_leaf(h->d_srch, h->d_leaf_cache, h->cache_np, pack_tree_bytes(m->D, narrow),
                         narrow ? 4 * L : L, h->num_sms, st);
    }
  } else if (m->kind == 2) {
    // MLP: set-up, prediction of c_profile, then predict + score all of TS
    const MlpDev md = m->mlp->dev();
    launch_mlp_prep(h->d_srch, h->d_steps, sb, st);
    launch_mlp_fwd(0, md, &h->d_steps[0].cprof_packed, 1, h->d_pcprof, nullptr, nullptr, nullptr,
                   nullptr, m->mlp->d_status, 1, st);
    mark(1);
    launch_mlp_fwd(1, md, h->space->d_packed, h->space->n_valid, h->d_s, h->d_pcprof, h->d_delta,
                   h->d_eval, h->d_mm, m->mlp->d_status, h->num_sms, st);
  } else if (m->kind == 3) {
    // least squares: set-up with c_profile's prediction, then predict + score TS
    launch_lsq_prep(h->d_srch, h->d_steps, sb, lsq_pack_bytes(m->lsq_m, m->lsq_nb, m->K), st);
    mark(1);
    launch_lsq_score(h->d_srch, m->lsq_m, m->lsq_nb, m->K, h->num_sms, st);
  } else {
    launch_bprep(h->d_srch, h->d_steps, sb, 1, m->K, m->D, st);
    mark(1);
    launch_bscore(h->d_srch, h->d_steps, h->d_items, h->n_items, h->mode,
                  h->opts.select == KTUNE_SELECT_TOPK, h->grid, st);
  }
  mark(2);
  if (h->opts.select == KTUNE_SELECT_SAMPLE) launch_bweights(h->d_srch, h->d_sub_search, h->n_sub, st);
  mark(3);
  launch_bselect(h->d_srch, h->d_steps, 1, st);
  mark(4);
}

// Capture the step into a graph once per (stream, timing mode); later steps
// only replace the prepare kernel's by-value step parameters and relaunch.
static int launch_step_graph(ktune_search *h, StepBatch<1> &sb, cudaStream_t st) {
  if (h->gexec && (h->graph_stream != st || h->graph_timing != h->timing)) drop_graph(h);
  if (!h->gexec) {
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    launch_step_kernels(h, sb, st, true);
    cudaGraph_t g = nullptr;
    CK(cudaStreamEndCapture(st, &g));
    h->graph = g;
    size_t n = 0;
    CK(cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    CK(cudaGraphGetNodes(g, nodes.data(), &n));
    for (cudaGraphNode_t nd : nodes) {
      cudaGraphNodeType t;
      CK(cudaGraphNodeGetType(nd, &t));
      if (t != cudaGraphNodeTypeKernel) continue;
      cudaKernelNodeParams kp{};
      CK(cudaGraphKernelNodeGetParams(nd, &kp));
      if (kp.func == bprep_func<1>() || kp.func == mlp_prep_func() || kp.func == lsq_prep_func() ||
          kp.func == nbr_score_func() || kp.func == table_prep_func())
        h->prep_node = nd;
    }
    if (!h->prep_node) FAIL(KTUNE_ECUDA, "graph capture lost the prepare kernel");
    CK(cudaGraphInstantiate(&h->gexec, g, 0));
    h->graph_stream = st;
    h->graph_timing = h->timing;
  } else {
    cudaKernelNodeParams kp{};
    CK(cudaGraphKernelNodeGetParams(h->prep_node, &kp));
    float *table = h->model->d_table;
    int64_t table_np = h->model->table_np;
    void *args[] = {&h->d_srch, &h->d_steps, &sb, &table, &table_np};
    kp.kernelParams = args;
    kp.extra = nullptr;
    CK(cudaGraphExecKernelNodeSetParams(h->gexec, h->prep_node, &kp));
  }
  CK(cudaGraphLaunch(h->gexec, st));
  return KTUNE_OK;
}

// A grid-barrier wait of the fused step that gave up (read and cleared).
static int fused_status(ktune_search *h) {
  if (!h->last_fused) return KTUNE_OK;
  int v = 0;
  CK(cudaMemcpy(&v, h->d_fz_status, 4, cudaMemcpyDeviceToHost));
  if (v) {
    CK(cudaMemset(h->d_fz_status, 0, 4));
    FAIL(KTUNE_ETIMEOUT, "a grid-barrier wait of the fused step timed out");
  }
  return KTUNE_OK;
}

static int enqueue_step(ktune_search *h, const float *counters, int k, int64_t *out_raw,
                        float *out_score, uint64_t *out_packed, int *n_out, cudaStream_t st,
                        int *status_out = nullptr) {
  StepBatch<1> sb{};
  StepDev &sp = sb.st[0];
  sp.cprof_packed = h->cprof_packed;
  host_expert(h->model->roles.data(), h->model->K, counters, h->opts.inst_reaction, h->opts.cores,
              sp.delta);
  sp.out_raw = out_raw;
  sp.out_score = out_score;
  sp.out_packed = out_packed;
  sp.n_out = n_out;
  sp.step = h->step_no;
  sp.k = k;
  h->last_fused = h->fused && !h->cached && !h->nbr_radius;
  if (h->last_fused) {
    // one cooperative launch: every CTA of the grid is resident at once
    FusedArgs fa{};
    fa.sd = h->sdh;
    fa.words = h->d_fz_words;
    fa.terms = h->d_fz_terms;
    fa.mm_live = h->d_fz_mm;
    fa.sync = h->d_fz_sync;
    fa.status = h->d_fz_status;
    fa.status_out = status_out;
    fa.cand = h->d_fz_cand;
    fa.list = h->d_fz_list;
    fa.wait_ns = 1000000000ull;
    fa.phase_ns = h->timing ? h->d_fz_phase : nullptr;
    fa.four = 4;
    fa.st = sp;
    if (h->timing) CK(cudaEventRecord(h->ev[0], st));
    CK(launch_step_fused(fa, h->fused - 1, h->opts.select == KTUNE_SELECT_TOPK, h->model->D,
                         h->fused_grid, st, h->mode == 2));
    if (h->timing) CK(cudaEventRecord(h->ev[1], st));
  } else if (st != nullptr && h->use_graph) {
    TRY(launch_step_graph(h, sb, st));
  } else {
    launch_step_kernels(h, sb, st, false);
  }
  CK(cudaGetLastError());
  h->last_stream = st;
  h->last_scored = h->space->n_valid - h->n_evaluated;
  h->step_no++;
  return KTUNE_OK;
}

int ktune_step(ktune_search *h, const float *counters, int k, int64_t *out_raw, float *out_score,
               int *n_out) {
  if (!h || !counters || !out_raw || !out_score || !n_out) FAIL(KTUNE_EINVAL, "null argument");
  if (k < 1 || k > KTUNE_MAX_K) FAIL(KTUNE_EINVAL, "k out of range");
  const int K = h->model->K;
  for (int i = 0; i < K; ++i)
    if (!isfinite(counters[i])) FAIL(KTUNE_EINVAL, "non-finite profiled counter");
  // the step's kernels write the outputs (and the fused step its barrier
  // status) into the mapped host block: no copies after the launch
  HostOut *ho = h->hout, *hd = h->hout_dev;
  ho->fused_status = 0;
  TRY(enqueue_step(h, counters, k, hd->raw, hd->score, hd->packed, &hd->n_out, h->stream,
                   &hd->fused_status));
  if (h->model->kind == 2)
    CK(cudaMemcpyAsync(h->h_nout + 1, h->model->mlp->d_status, 4, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->model->kind == 2 && h->h_nout[1]) {
    cudaMemset(h->model->mlp->d_status, 0, 4);
    FAIL(KTUNE_ETIMEOUT, "a tensor-core wait of the MLP timed out");
  }
  if (h->last_fused && ho->fused_status) FAIL(KTUNE_ETIMEOUT, "a grid-barrier wait of the fused step timed out");
  const int n = ho->n_out;
  *n_out = n;
  memcpy(out_raw, ho->raw, n * 8);
  memcpy(out_score, ho->score, n * 4);
  h->last_raw.assign(ho->raw, ho->raw + n);
  h->last_packed.assign(ho->packed, ho->packed + n);
  h->n_evaluated += n;
  if (h->nbr_radius) {
    if (n == 0) FAIL(KTUNE_EXHAUSTED, "no unevaluated valid configuration in the neighbourhood");
    return KTUNE_OK;
  }
  if (n < k) FAIL(KTUNE_EXHAUSTED, "fewer unevaluated configurations than requested");
  return KTUNE_OK;
}

int ktune_step_device(ktune_search *h, const float *counters, int k, int64_t *out_raw_dev,
                      float *out_score_dev, int *n_out_dev, void *stream) {
  if (!h || !counters || !out_raw_dev || !out_score_dev) FAIL(KTUNE_EINVAL, "null argument");
  if (k < 1 || k > KTUNE_MAX_K) FAIL(KTUNE_EINVAL, "k out of range");
  for (int i = 0; i < h->model->K; ++i)
    if (!isfinite(counters[i])) FAIL(KTUNE_EINVAL, "non-finite profiled counter");
  h->last_raw.clear();
  h->last_packed.clear();
  TRY(enqueue_step(h, counters, k, out_raw_dev, out_score_dev, h->d_out_packed, n_out_dev,
                   (cudaStream_t)stream));
  // the number drawn is known only on the device; it is k unless the space ran out
  h->n_evaluated = std::min<int64_t>(h->space->n_valid, h->n_evaluated + k);
  return KTUNE_OK;
}

// ---- checkpoints -------------------------------------------------------------
// Blob (little-endian): header, then the last returned batch (raw indices,
// packed digits) awaiting ktune_report, then the evaluated bitset words.
namespace {
constexpr uint32_t kCkptMagic = 0x4B50434Bu;   // "KCPK"
constexpr uint32_t kCkptVersion = 1;
struct CkptHeader {
  uint32_t magic, version;
  int64_t n_valid, n_raw;
  int32_t n_params, K, depth, kind;
  ktune_search_opts opts;
  int64_t cprof_raw;
  int64_t n_evaluated;
  uint32_t step_no;
  int32_t n_last;
  uint64_t space_hash;      // FNV-1a over the radices and the constraint table
};

uint64_t space_hash(const ktune_space *s) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](const void *p, size_t n) {
    const uint8_t *b = static_cast<const uint8_t *>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  };
  mix(s->sa.radix, sizeof(int) * s->sa.P);
  mix(s->values.data(), s->values.size() * sizeof(int64_t));
  mix(s->table.data(), s->table.size() * sizeof(uint32_t));
  return h;
}

size_t ckpt_bytes(const ktune_search *h, size_t n_last) {
  return sizeof(CkptHeader) + n_last * 16 + (size_t)((h->space->n_valid + 31) / 32) * 4;
}
}  // namespace

int ktune_search_save(const ktune_search *h, void *buf, size_t *bytes) {
  if (!h || !bytes) FAIL(KTUNE_EINVAL, "null argument");
  const size_t need = ckpt_bytes(h, h->last_raw.size());
  if (!buf) {
    *bytes = need;
    return KTUNE_OK;
  }
  if (*bytes < need) {
    *bytes = need;
    FAIL(KTUNE_EINVAL, "checkpoint buffer too small");
  }
  CkptHeader hd{};
  hd.magic = kCkptMagic;
  hd.version = kCkptVersion;
  hd.n_valid = h->space->n_valid;
  hd.n_raw = h->space->sa.n_raw;
  hd.n_params = h->space->sa.P;
  hd.K = h->model->K;
  hd.depth = h->model->D;
  hd.kind = h->model->kind;
  hd.opts = h->opts;
  hd.cprof_raw = h->cprof_raw;
  hd.n_evaluated = h->n_evaluated;
  hd.step_no = h->step_no;
  hd.n_last = (int32_t)h->last_raw.size();
  hd.space_hash = space_hash(h->space);
  uint8_t *p = static_cast<uint8_t *>(buf);
  memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  if (hd.n_last) {
    memcpy(p, h->last_raw.data(), (size_t)hd.n_last * 8);
    memcpy(p + (size_t)hd.n_last * 8, h->last_packed.data(), (size_t)hd.n_last * 8);
  }
  p += (size_t)hd.n_last * 16;
  const size_t words = (size_t)((h->space->n_valid + 31) / 32);
  // the state includes every step enqueued so far
  CK(cudaStreamSynchronize(h->last_stream ? h->last_stream : h->stream));
  CK(cudaMemcpy(p, h->d_eval, words * 4, cudaMemcpyDeviceToHost));
  *bytes = need;
  return KTUNE_OK;
}

int ktune_search_load(ktune_space *s, ktune_model *m, const void *buf, size_t bytes, void *stream,
                      ktune_search **out) {
  if (!s || !m || !buf || !out) FAIL(KTUNE_EINVAL, "null argument");
  *out = nullptr;
  CkptHeader hd;
  if (bytes < sizeof(hd)) FAIL(KTUNE_EINVAL, "checkpoint truncated");
  memcpy(&hd, buf, sizeof(hd));
  if (hd.magic != kCkptMagic || hd.version != kCkptVersion) FAIL(KTUNE_EINVAL, "not a search checkpoint");
  if (hd.n_valid != s->n_valid || hd.n_raw != s->sa.n_raw || hd.n_params != s->sa.P ||
      hd.space_hash != space_hash(s))
    FAIL(KTUNE_EINVAL, "checkpoint belongs to another tuning space");
  if (hd.K != m->K || hd.depth != m->D || hd.kind != m->kind)
    FAIL(KTUNE_EMODEL, "checkpoint belongs to another model");
  if (hd.n_last < 0 || hd.n_last > KTUNE_MAX_K || hd.n_evaluated < 1 || hd.n_evaluated > s->n_valid ||
      hd.cprof_raw < 0 || hd.cprof_raw >= s->sa.n_raw)
    FAIL(KTUNE_EINVAL, "checkpoint fields out of range");
  ktune_search *h = nullptr;
  const size_t need = sizeof(hd) + (size_t)hd.n_last * 16 + (size_t)((s->n_valid + 31) / 32) * 4;
  if (bytes < need) FAIL(KTUNE_EINVAL, "checkpoint truncated");
  TRY(ktune_search_create(s, m, &hd.opts, stream, &h));
  const uint8_t *p = static_cast<const uint8_t *>(buf) + sizeof(hd);
  h->last_raw.assign(reinterpret_cast<const int64_t *>(p), reinterpret_cast<const int64_t *>(p) + hd.n_last);
  h->last_packed.assign(reinterpret_cast<const uint64_t *>(p + (size_t)hd.n_last * 8),
                        reinterpret_cast<const uint64_t *>(p + (size_t)hd.n_last * 8) + hd.n_last);
  p += (size_t)hd.n_last * 16;
  const size_t words = (size_t)((s->n_valid + 31) / 32);
  if (cudaMemcpyAsync(h->d_eval, p, words * 4, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    ktune_search_destroy(h);
    FAIL(KTUNE_ECUDA, "checkpoint upload failed");
  }
  h->cprof_raw = hd.cprof_raw;
  h->cprof_packed = host_pack(s, hd.cprof_raw);
  h->n_evaluated = hd.n_evaluated;
  h->step_no = hd.step_no;
  *out = h;
  return KTUNE_OK;
}

int ktune_search_set_neighbourhood(ktune_search *h, int radius) {
  if (!h) FAIL(KTUNE_EINVAL, "null search");
  if (radius < 0 || radius > 2) FAIL(KTUNE_EINVAL, "neighbourhood radius must be 0, 1 or 2");
  const ktune_space *s = h->space;
  if (radius && (!s->d_packed || h->model->kind != 1))
    FAIL(KTUNE_ESTATE, "neighbourhood steps need a materialised space and a tree model");
  NbrDev nb{};
  const int P = s->sa.P;
  int64_t C1 = 0, C2 = 0;
  if (radius) {
    nb.radius = radius;
    for (int j = 0; j < P; ++j) {
      nb.radix_m1[j] = s->sa.radix[j] - 1;
      nb.off1[j] = (int)C1;
      C1 += nb.radix_m1[j];
    }
    nb.off1[P] = (int)C1;
    int q = 0;
    if (radius == 2)
      for (int i = 0; i < P; ++i)
        for (int j = i + 1; j < P; ++j) {
          nb.pi[q] = (uint8_t)i;
          nb.pj[q] = (uint8_t)j;
          nb.off2[q] = (int)C2;
          C2 += (int64_t)nb.radix_m1[i] * nb.radix_m1[j];
          ++q;
        }
    nb.off2[q] = (int)C2;
    nb.n_pairs = q;
    if (C1 + C2 > kNbrMaxCandidates) FAIL(KTUNE_EINVAL, "neighbourhood larger than 2^20 configurations");
    nb.C1 = (int)C1;
    nb.C = (int)(C1 + C2);
  }
  CK(cudaStreamSynchronize(h->last_stream ? h->last_stream : h->stream));
  cudaFree(h->d_nbr);
  cudaFree(h->d_nbr_buf);
  h->d_nbr = nullptr;
  h->d_nbr_buf = nullptr;
  h->nbr_radius = 0;
  h->nbr_C = 0;
  h->sdh.nbr = nullptr;
  if (radius) {
    const size_t C = (size_t)std::max(1, nb.C);
    // per candidate: ord_e 4 + s_e 4 + p_e 8; compacted: ord 4 + s 4 + p 8 + w 8; count
    const size_t bytes = C * (4 + 4 + 8) + C * (4 + 4 + 8 + 8) + 256;
    int rc;
    if ((rc = dalloc(&h->d_nbr_buf, bytes)) || (rc = dalloc(&h->d_nbr, 1))) return rc;
    uint8_t *b = h->d_nbr_buf;
    nb.p_e = reinterpret_cast<uint64_t *>(b); b += C * 8;
    nb.p = reinterpret_cast<uint64_t *>(b); b += C * 8;
    nb.w = reinterpret_cast<uint64_t *>(b); b += C * 8;
    nb.ord_e = reinterpret_cast<uint32_t *>(b); b += C * 4;
    nb.s_e = reinterpret_cast<float *>(b); b += C * 4;
    nb.ord = reinterpret_cast<uint32_t *>(b); b += C * 4;
    nb.s = reinterpret_cast<float *>(b); b += C * 4;
    nb.count = reinterpret_cast<int *>(b);
    CK(cudaMemcpy(h->d_nbr, &nb, sizeof(nb), cudaMemcpyHostToDevice));
    CK(cudaMemset(nb.count, 0, 4));
    h->nbr_radius = radius;
    h->nbr_C = nb.C;
    h->sdh.nbr = h->d_nbr;
  }
  CK(cudaMemcpy(h->d_srch, &h->sdh, sizeof(SearchDev), cudaMemcpyHostToDevice));
  drop_graph(h);
  return KTUNE_OK;
}

// Whether the least-squares prepare kernel writes the register kernel's pack
// (cached steps read prediction columns instead).
static int set_lsq_pack(ktune_search *h, bool on) {
  if (h->model->kind != 3 || h->sdh.lsq_pack == (int)on) return KTUNE_OK;
  h->sdh.lsq_pack = on;
  CK(cudaMemcpy(&h->d_srch->lsq_pack, &h->sdh.lsq_pack, sizeof(int), cudaMemcpyHostToDevice));
  return KTUNE_OK;
}

int ktune_search_set_cached(ktune_search *h, int enable) {
  if (!h) FAIL(KTUNE_EINVAL, "null search");
  if (enable && h->model->kind == 4)
    FAIL(KTUNE_ESTATE, "a counter-table model is scored from its table already");
  if (!enable) {
    if (h->cached || h->d_cache || h->d_leaf_cache) {
      CK(cudaStreamSynchronize(h->last_stream ? h->last_stream : h->stream));
      cudaFree(h->d_cache);
      cudaFree(h->d_leaf_cache);
      h->d_cache = nullptr;
      h->d_leaf_cache = nullptr;
      h->cached = false;
      drop_graph(h);
      TRY(set_lsq_pack(h, h->model->kind == 3));
    }
    return KTUNE_OK;
  }
  const ktune_space *s = h->space;
  if (!s->d_packed) FAIL(KTUNE_ESTATE, "cached predictions need a materialised space");
  if (h->opts.select != KTUNE_SELECT_SAMPLE) FAIL(KTUNE_ESTATE, "cached predictions need weighted-draw selection");
  const int K = h->model->K;
  const int64_t N = s->n_valid, Np = (N + 7) & ~(int64_t)7;
  cudaStream_t st = h->stream;
  CK(cudaStreamSynchronize(h->last_stream ? h->last_stream : st));
  if (h->model->kind == 1) {   // trees: the leaf index of every configuration in every tree
    if (!h->d_leaf_cache) {
      int rc = dalloc(&h->d_leaf_cache, (size_t)K * Np);
      if (rc) return rc;
      h->cache_np = Np;
    }
    launch_leaf_cols(s->d_packed, N, h->model->d_nodes, K, h->model->D, h->d_leaf_cache, Np, st);
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) FAIL(KTUNE_ECUDA, std::string("cache fill: ") + cudaGetErrorString(e));
    h->cached = true;
    drop_graph(h);
    return KTUNE_OK;
  }
  if (!h->d_cache) {
    int rc = dalloc(&h->d_cache, (size_t)K * Np);
    if (rc) return rc;
    h->cache_np = Np;
  }
  // predictions in chunks of rows, each transposed into the columns
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(N, (int64_t)(16 << 20) / K));
  float *rows = nullptr;
  int rc = dalloc(&rows, (size_t)chunk * K);
  if (rc) return rc;
  for (int64_t first = 0; first < N && rc == KTUNE_OK; first += chunk) {
    const int64_t n = std::min<int64_t>(chunk, N - first);
    rc = ktune_model_predict_device(h->model, first, n, rows, st);
    if (rc == KTUNE_OK) launch_rows_to_cols(rows, n, K, h->d_cache, Np, first, st);
  }
  const cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(rows);
  if (rc) return rc;
  if (e != cudaSuccess) FAIL(KTUNE_ECUDA, std::string("cache fill: ") + cudaGetErrorString(e));
  if (h->model->kind == 2) {
    int status = 0;
    CK(cudaMemcpy(&status, h->model->mlp->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status) {
      cudaMemset(h->model->mlp->d_status, 0, sizeof(int));
      FAIL(KTUNE_ETIMEOUT, "a tensor-core wait of the MLP timed out");
    }
  }
  TRY(set_lsq_pack(h, false));
  h->cached = true;
  drop_graph(h);
  return KTUNE_OK;
}

int ktune_search_set_timing(ktune_search *h, int enable) {
  if (!h) FAIL(KTUNE_EINVAL, "null search");
  if (enable && !h->ev[0])
    for (auto &e : h->ev) CK(cudaEventCreate(&e));
  h->timing = enable != 0;
  return KTUNE_OK;
}

int ktune_search_stats(ktune_search *h, ktune_step_stats *out) {
  if (!h || !out) FAIL(KTUNE_EINVAL, "null argument");
  memset(out, 0, sizeof(*out));
  CK(cudaStreamSynchronize(h->last_stream));
  int na = 0;
  int mm[2] = {0, 0};
  CK(cudaMemcpy(&na, h->d_nactive, 4, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(mm, h->d_mm, 8, cudaMemcpyDeviceToHost));
  auto inv = [](int k) {
    const int b = k >= 0 ? k : k ^ 0x7FFFFFFF;
    float f;
    memcpy(&f, &b, 4);
    return f;
  };
  out->n_scored = h->last_scored;
  if (h->nbr_radius) {
    int nc = 0;
    NbrDev nb;
    CK(cudaMemcpy(&nb, h->d_nbr, sizeof(nb), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&nc, nb.count, 4, cudaMemcpyDeviceToHost));
    out->n_scored = nc;
  }
  out->n_active = na;
  out->depth = h->model->D;
  const bool none = mm[0] == 0x7FFFFFFF && mm[1] == (int)0x80000000;
  out->s_min = none ? INFINITY : inv(mm[0]);
  out->s_max = none ? -INFINITY : inv(mm[1]);
  if (h->timing && h->last_fused) {
    out->n_kernels = 1;
    CK(cudaEventElapsedTime(&out->kernel_ms[0], h->ev[0], h->ev[1]));
    // the fused kernel's phases, from its time stamps
    uint64_t t[8];
    CK(cudaMemcpy(t, h->d_fz_phase, sizeof(t), cudaMemcpyDeviceToHost));
    const bool sample = h->opts.select == KTUNE_SELECT_SAMPLE;
    const uint64_t end_p1 = sample ? t[3] : t[5];
    const double ph[7] = {(double)(t[1] - t[0]), (double)(t[2] - t[1]), (double)(end_p1 - t[2]),
                          sample ? (double)(t[4] - t[3]) : 0.0, sample ? (double)(t[5] - t[4]) : 0.0,
                          (double)((int64_t)(t[6] - t[5])), (double)(t[7] - t[6])};
    for (int i = 0; i < 7; ++i) out->kernel_ms[1 + i] = (float)(ph[i] * 1e-6);
  } else if (h->timing) {
    out->n_kernels = 4;
    for (int i = 0; i < 4; ++i) CK(cudaEventElapsedTime(&out->kernel_ms[i], h->ev[i], h->ev[i + 1]));
  }
  TRY(fused_status(h));
  return KTUNE_OK;
}

int ktune_search_set_fused(ktune_search *h, int shape) {
  if (!h) FAIL(KTUNE_EINVAL, "null search");
  if (shape < 0 || shape > fused_shapes()) FAIL(KTUNE_EINVAL, "unknown fused-kernel shape");
  if (shape > 0 && !h->d_fz_words)
    FAIL(KTUNE_ESTATE, "the fused step needs a tree model on a one-word space");
  if (shape > 0 && fused_blocks_per_sm(shape - 1) < 1)
    FAIL(KTUNE_ESTATE, "this kernel shape cannot be resident on this device");
  if (shape > 0 && h->mode == 2 && shape != 2)
    FAIL(KTUNE_ESTATE, "on-the-fly spaces take the fused step in shape 2 only");
  CK(cudaStreamSynchronize(h->last_stream));
  h->fused = shape;
  return KTUNE_OK;
}

int ktune_search_scores_device(const ktune_search *h, int64_t first, int64_t count,
                               float *scores_dev, uint32_t *weights_dev, void *stream) {
  if (!h || (!scores_dev && !weights_dev)) FAIL(KTUNE_EINVAL, "null argument");
  const int64_t N = h->space->n_valid;
  if (first < 0 || count < 0 || first > N || count > N - first) FAIL(KTUNE_EINVAL, "range out of TS");
  if (h->nbr_radius) FAIL(KTUNE_ESTATE, "neighbourhood-restricted steps score only their candidates");
  if (weights_dev && h->opts.select != KTUNE_SELECT_SAMPLE)
    FAIL(KTUNE_ESTATE, "top-k searches compute no weights");
  if (count == 0) return KTUNE_OK;
  const cudaStream_t st = (cudaStream_t)stream;
  if (scores_dev)
    CK(cudaMemcpyAsync(scores_dev, h->d_s + first, (size_t)count * 4, cudaMemcpyDeviceToDevice, st));
  if (weights_dev)
    CK(cudaMemcpyAsync(weights_dev, h->d_w + first, (size_t)count * 4, cudaMemcpyDeviceToDevice, st));
  return KTUNE_OK;
}

int ktune_report(ktune_search *h, const double *runtimes, int n) {
  if (!h || (!runtimes && n)) FAIL(KTUNE_EINVAL, "null argument");
  if (n != (int)h->last_raw.size() || n == 0) FAIL(KTUNE_ESTATE, "no matching ktune_step to report");
  double t = INFINITY;
  for (int i = 0; i < n; ++i) {
    if (isnan(runtimes[i])) FAIL(KTUNE_EINVAL, "NaN runtime");
    if (runtimes[i] <= t) {
      t = runtimes[i];
      h->cprof_raw = h->last_raw[i];
      h->cprof_packed = h->last_packed[i];
    }
  }
  h->last_raw.clear();
  h->last_packed.clear();
  return KTUNE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched steps
namespace {

struct BatchVariant {
  int score_variant, items_per_cta;
};
const BatchVariant kBatchVariants[] = {{0, 1}, {0, 4}, {1, 1}, {2, 1}, {2, 4}, {3, 1}, {4, 1}, {4, 4}};
constexpr int kNumBatchVariants = sizeof(kBatchVariants) / sizeof(kBatchVariants[0]);

// Work items of the batch: every search's space (ordinals, or raw tiles when on
// the fly) cut into pieces of about total / (SMs * items_per_cta) units.
int batch_items(ktune_batch *b) {
  std::vector<ItemDev> items;
  int64_t total = 0;
  for (ktune_search *h : b->s)
    if (h->model->kind != 2) total += b->mode == 2 ? h->space->n_tiles : h->space->n_valid;
  const int64_t target =
      std::max<int64_t>(b->mode == 2 ? 1 : 1024, total / ((int64_t)b->num_sms * b->items_per_cta));
  for (size_t i = 0; i < b->s.size(); ++i) {
    ktune_search *h = b->s[i];
    b->sdh[i].item_begin = (int64_t)items.size();
    if (h->model->kind == 2) {   // scored by the MLP kernels, no tree-walk items
      b->sdh[i].item_end = (int64_t)items.size();
      continue;
    }
    const int64_t units = b->mode == 2 ? h->space->n_tiles : h->space->n_valid;
    const int64_t pieces = std::max<int64_t>(1, (units + target - 1) / target);
    for (int64_t q = 0; q < pieces; ++q) {
      ItemDev it{};
      it.search = (int)i;
      it.lo = units * q / pieces;
      it.hi = units * (q + 1) / pieces;
      if (it.hi > it.lo) items.push_back(it);
    }
    b->sdh[i].item_end = (int64_t)items.size();
  }
  b->n_items = (int)items.size();
  b->grid = std::min<int>(b->n_items, b->num_sms);
  cudaFree(b->d_items);
  cudaFree(b->d_cand_key);
  cudaFree(b->d_cand_raw);
  b->d_items = nullptr;
  b->d_cand_key = nullptr;
  b->d_cand_raw = nullptr;
  int rc;
  const size_t n_alloc = std::max<size_t>(1, items.size());
  if ((rc = dalloc(&b->d_items, n_alloc)) || (rc = dalloc(&b->d_cand_key, n_alloc * KTUNE_MAX_K)) ||
      (rc = dalloc(&b->d_cand_raw, n_alloc * KTUNE_MAX_K)))
    return rc;
  for (size_t i = 0; i < b->s.size(); ++i) {
    // candidates of search i live after those of the searches before it; the
    // kernels index them by (item - item_begin)
    b->sdh[i].cand_key = b->d_cand_key + b->sdh[i].item_begin * KTUNE_MAX_K;
    b->sdh[i].cand_raw = b->d_cand_raw + b->sdh[i].item_begin * KTUNE_MAX_K;
  }
  if (!items.empty())
    CK(cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(ItemDev),
                       cudaMemcpyHostToDevice, b->stream));
  CK(cudaMemcpyAsync(b->d_srch, b->sdh.data(), b->sdh.size() * sizeof(SearchDev),
                     cudaMemcpyHostToDevice, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  return KTUNE_OK;
}

void batch_drop_graph(ktune_batch *b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
  b->prep_node = nullptr;
}

int batch_fill_steps(ktune_batch *b, const float *const *counters, int k, StepBatch<kMaxBatch> &sb) {
  for (size_t i = 0; i < b->s.size(); ++i) {
    ktune_search *h = b->s[i];
    const int K = h->model->K;
    if (!counters[i]) FAIL(KTUNE_EINVAL, "null counters");
    for (int q = 0; q < K; ++q)
      if (!isfinite(counters[i][q])) FAIL(KTUNE_EINVAL, "non-finite profiled counter");
    StepDev &sp = sb.st[i];
    sp.cprof_packed = h->cprof_packed;
    host_expert(h->model->roles.data(), K, counters[i], h->opts.inst_reaction, h->opts.cores,
                sp.delta);
    sp.out_raw = b->d_out_raw + i * KTUNE_MAX_K;
    sp.out_score = b->d_out_score + i * KTUNE_MAX_K;
    sp.out_packed = b->d_out_packed + i * KTUNE_MAX_K;
    sp.n_out = b->d_nout + i;
    sp.step = h->step_no;
    sp.k = k;
  }
  return KTUNE_OK;
}

void batch_launch(ktune_batch *b, const StepBatch<kMaxBatch> &sb, cudaStream_t st, bool score_only) {
  const int S = (int)b->s.size();
  launch_bprep<kMaxBatch>(b->d_srch, b->d_steps, sb, S, b->K_max, b->D_max, st);
  if (b->n_items > 0)
    launch_bscore(b->d_srch, b->d_steps, b->d_items, b->n_items, b->mode, b->topk, b->grid, st,
                  b->variant);
  if (score_only) return;
  // searches scored by the MLP: prediction of c_profile, then the fused
  // tensor-core forward + Eq. score over all of TS (the same kernels as a
  // single MLP step)
  for (const auto &g : b->mlp_groups) {
    const ktune_search *h = g.first;
    const MlpDev md = h->model->mlp->dev();
    const int S = (int)g.members.size();
    launch_mlp_fwd(0, md, g.d_cprof, S, g.d_pcprof, nullptr, nullptr, nullptr, nullptr,
                   h->model->mlp->d_status, 1, st);
    launch_mlp_score_shared(md, h->space->d_packed, h->space->n_valid, g.tg,
                            h->model->mlp->d_status, b->num_sms, st);
  }
  if (!b->topk) launch_bweights(b->d_srch, b->d_sub_search, b->n_sub, st);
  launch_bselect(b->d_srch, b->d_steps, S, st);
}

}  // namespace

extern "C" {

int ktune_batch_variant(int v, int *threads, int *cpt, int *items_per_cta) {
  if (v >= 0 && v < kNumBatchVariants) {
    if (threads) *threads = bscore_variant_threads(kBatchVariants[v].score_variant);
    if (cpt) *cpt = bscore_variant_cpt(kBatchVariants[v].score_variant);
    if (items_per_cta) *items_per_cta = kBatchVariants[v].items_per_cta;
  }
  return kNumBatchVariants;
}

int ktune_batch_create(ktune_search *const *searches, int n, void *stream, ktune_batch **out) {
  if (!searches || !out || n < 1) FAIL(KTUNE_EINVAL, "null argument or empty batch");
  if (n > kMaxBatch) FAIL(KTUNE_EINVAL, "more than 64 searches in a batch");
  *out = nullptr;
  int tree0 = -1;   // first search scored by trees (its space mode is the batch's)
  for (int i = 0; i < n; ++i) {
    if (!searches[i]) FAIL(KTUNE_EINVAL, "null search");
    if (searches[i]->opts.select != searches[0]->opts.select)
      FAIL(KTUNE_EINVAL, "searches of a batch must share the select mode");
    if (searches[i]->model->kind == 1 && tree0 < 0) tree0 = i;
    if (searches[i]->model->kind == 3) FAIL(KTUNE_EINVAL, "least-squares searches step on their own");
    if (searches[i]->model->kind == 4) FAIL(KTUNE_EINVAL, "counter-table searches step on their own");
    if (searches[i]->nbr_radius) FAIL(KTUNE_EINVAL, "neighbourhood-restricted searches step on their own");
  }
  for (int i = 0; i < n; ++i)
    if (searches[i]->model->kind == 1 && searches[i]->mode != searches[tree0]->mode)
      FAIL(KTUNE_EINVAL, "tree-scored searches of a batch must share the space mode");
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j)
      if (searches[i] == searches[j]) FAIL(KTUNE_EINVAL, "a search appears twice in the batch");
  ktune_batch *b = new (std::nothrow) ktune_batch();
  if (!b) FAIL(KTUNE_ENOMEM, "host allocation");
  auto fail = [&](int rc) {
    ktune_batch_destroy(b);
    return rc;
  };
  b->s.assign(searches, searches + n);
  b->mode = tree0 >= 0 ? searches[tree0]->mode : 0;
  b->topk = searches[0]->opts.select == KTUNE_SELECT_TOPK;
  b->stream = (cudaStream_t)stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
  std::vector<int> sub_search;
  for (int i = 0; i < n; ++i) {
    ktune_search *h = searches[i];
    b->K_max = std::max(b->K_max, h->model->K);
    if (h->model->kind == 1) b->D_max = std::max(b->D_max, h->model->D);
    SearchDev sd = h->sdh;
    sd.sub_begin = (int64_t)sub_search.size();
    for (int64_t g = 0; g < h->n_sub; ++g) sub_search.push_back(i);
    b->sdh.push_back(sd);
  }
  b->n_sub = (int64_t)sub_search.size();
  int rc;
  for (int i = 0; i < n; ++i) {
    ktune_search *h = searches[i];
    if (h->model->kind != 2) continue;
    ktune_batch::MlpGroup *g = nullptr;
    for (auto &e : b->mlp_groups)
      if (e.first->model->mlp == h->model->mlp && e.first->space == h->space &&
          (int)e.members.size() < kMlpMaxShare)
        g = &e;
    if (!g) {
      b->mlp_groups.emplace_back();
      g = &b->mlp_groups.back();
      g->first = h;
    }
    g->members.push_back(i);
  }
  for (auto &g : b->mlp_groups) {
    const int S = (int)g.members.size(), K = g.first->model->K;
    if ((rc = dalloc(&g.d_cprof, S)) || (rc = dalloc(&g.d_pcprof, (size_t)S * K))) return fail(rc);
    g.tg.S = S;
    for (int q = 0; q < S; ++q) {
      ktune_search *m = searches[g.members[q]];
      b->sdh[g.members[q]].cprof_slot = g.d_cprof + q;
      g.tg.pcprof[q] = g.d_pcprof + (size_t)q * K;
      g.tg.delta[q] = m->d_delta;
      g.tg.s[q] = m->d_s;
      g.tg.eval[q] = m->d_eval;
      g.tg.mm[q] = m->d_mm;
    }
  }
  if ((rc = dalloc(&b->d_srch, n)) || (rc = dalloc(&b->d_steps, n)) ||
      (rc = dalloc(&b->d_sub_search, sub_search.size())) ||
      (rc = dalloc(&b->d_out_raw, (size_t)n * KTUNE_MAX_K)) ||
      (rc = dalloc(&b->d_out_score, (size_t)n * KTUNE_MAX_K)) ||
      (rc = dalloc(&b->d_out_packed, (size_t)n * KTUNE_MAX_K)) || (rc = dalloc(&b->d_nout, n)))
    return fail(rc);
  if (cudaMallocHost((void **)&b->h_out_raw, (size_t)n * KTUNE_MAX_K * 8) != cudaSuccess ||
      cudaMallocHost((void **)&b->h_out_score, (size_t)n * KTUNE_MAX_K * 4) != cudaSuccess ||
      cudaMallocHost((void **)&b->h_out_packed, (size_t)n * KTUNE_MAX_K * 8) != cudaSuccess ||
      cudaMallocHost((void **)&b->h_nout, (size_t)n * 4) != cudaSuccess) {
    set_error("pinned host allocation failed");
    return fail(KTUNE_ENOMEM);
  }
  if (cudaMemcpyAsync(b->d_sub_search, sub_search.data(), sub_search.size() * 4,
                      cudaMemcpyHostToDevice, b->stream) != cudaSuccess) {
    set_error("upload failed");
    return fail(KTUNE_ECUDA);
  }
  if ((rc = batch_items(b))) return fail(rc);
  *out = b;
  return KTUNE_OK;
}

int ktune_batch_destroy(ktune_batch *b) {
  if (!b) return KTUNE_OK;
  void *dev[] = {b->d_srch, b->d_steps, b->d_items, b->d_sub_search, b->d_cand_key, b->d_cand_raw,
                 b->d_out_raw, b->d_out_score, b->d_out_packed, b->d_nout};
  for (void *p : dev) cudaFree(p);
  void *pin[] = {b->h_out_raw, b->h_out_score, b->h_out_packed, b->h_nout};
  for (void *p : pin) cudaFreeHost(p);
  for (auto &g : b->mlp_groups) {
    cudaFree(g.d_cprof);
    cudaFree(g.d_pcprof);
  }
  batch_drop_graph(b);
  delete b;
  return KTUNE_OK;
}

int ktune_batch_step(ktune_batch *b, const float *const *counters, int k, int64_t *out_raw,
                     float *out_score, int *n_out) {
  if (!b || !counters || !out_raw || !out_score || !n_out) FAIL(KTUNE_EINVAL, "null argument");
  if (k < 1 || k > KTUNE_MAX_K) FAIL(KTUNE_EINVAL, "k out of range");
  static thread_local StepBatch<kMaxBatch> sb;
  memset(&sb, 0, sizeof(sb));
  TRY(batch_fill_steps(b, counters, k, sb));
  const int S = (int)b->s.size();
  cudaStream_t st = b->stream;
  if (st) {
    if (b->gexec && b->graph_stream != st) batch_drop_graph(b);
    if (!b->gexec) {
      CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      batch_launch(b, sb, st, false);
      cudaGraph_t g = nullptr;
      CK(cudaStreamEndCapture(st, &g));
      b->graph = g;
      size_t nn = 0;
      CK(cudaGraphGetNodes(g, nullptr, &nn));
      std::vector<cudaGraphNode_t> nodes(nn);
      CK(cudaGraphGetNodes(g, nodes.data(), &nn));
      for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        CK(cudaGraphNodeGetType(nd, &t));
        if (t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp{};
        CK(cudaGraphKernelNodeGetParams(nd, &kp));
        if (kp.func == bprep_func<kMaxBatch>()) b->prep_node = nd;
      }
      if (!b->prep_node) FAIL(KTUNE_ECUDA, "graph capture lost the prepare kernel");
      CK(cudaGraphInstantiate(&b->gexec, g, 0));
      b->graph_stream = st;
    } else {
      cudaKernelNodeParams kp{};
      CK(cudaGraphKernelNodeGetParams(b->prep_node, &kp));
      void *args[] = {&b->d_srch, &b->d_steps, &sb};
      kp.kernelParams = args;
      kp.extra = nullptr;
      CK(cudaGraphExecKernelNodeSetParams(b->gexec, b->prep_node, &kp));
    }
    CK(cudaGraphLaunch(b->gexec, st));
  } else {
    batch_launch(b, sb, st, false);
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(b->h_out_raw, b->d_out_raw, (size_t)S * KTUNE_MAX_K * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(b->h_out_score, b->d_out_score, (size_t)S * KTUNE_MAX_K * 4, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(b->h_out_packed, b->d_out_packed, (size_t)S * KTUNE_MAX_K * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(b->h_nout, b->d_nout, (size_t)S * 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (ktune_search *h : b->s)
    if (h->model->kind == 2) {
      int status = 0;
      CK(cudaMemcpy(&status, h->model->mlp->d_status, sizeof(int), cudaMemcpyDeviceToHost));
      if (status) {
        cudaMemset(h->model->mlp->d_status, 0, sizeof(int));
        FAIL(KTUNE_ETIMEOUT, "a tensor-core wait of the MLP timed out");
      }
    }
  bool exhausted = false;
  for (int i = 0; i < S; ++i) {
    ktune_search *h = b->s[i];
    const int no = b->h_nout[i];
    n_out[i] = no;
    exhausted |= no < k;
    for (int j = 0; j < no; ++j) {
      out_raw[(size_t)i * k + j] = b->h_out_raw[(size_t)i * KTUNE_MAX_K + j];
      out_score[(size_t)i * k + j] = b->h_out_score[(size_t)i * KTUNE_MAX_K + j];
    }
    h->last_raw.assign(b->h_out_raw + (size_t)i * KTUNE_MAX_K, b->h_out_raw + (size_t)i * KTUNE_MAX_K + no);
    h->last_packed.assign(b->h_out_packed + (size_t)i * KTUNE_MAX_K,
                          b->h_out_packed + (size_t)i * KTUNE_MAX_K + no);
    h->last_scored = h->space->n_valid - h->n_evaluated;
    h->n_evaluated += no;
    h->step_no++;
    h->last_stream = st;
  }
  if (exhausted) FAIL(KTUNE_EXHAUSTED, "a search has fewer unevaluated configurations than requested");
  return KTUNE_OK;
}

int ktune_batch_autotune(ktune_batch *b, const float *const *counters, int reps, int *choice,
                         float *ms_out, int n_ms) {
  if (!b || !counters || reps < 1) FAIL(KTUNE_EINVAL, "bad argument");
  static thread_local StepBatch<kMaxBatch> sb;
  memset(&sb, 0, sizeof(sb));
  TRY(batch_fill_steps(b, counters, 1, sb));
  cudaStream_t st = b->stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int best = 0;
  float best_ms = INFINITY;
  const int nv = b->mode == 2 ? 1 : kNumBatchVariants;   // on-the-fly spaces have one shape
  for (int v = 0; v < nv; ++v) {
    b->variant = kBatchVariants[v].score_variant;
    b->items_per_cta = kBatchVariants[v].items_per_cta;
    TRY(batch_items(b));
    batch_launch(b, sb, st, true);   // warm-up (scoring only: no search state changes)
    CK(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r) batch_launch(b, sb, st, true);
    CK(cudaEventRecord(e1, st));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    ms /= reps;
    if (ms_out && v < n_ms) ms_out[v] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->variant = kBatchVariants[best].score_variant;
  b->items_per_cta = kBatchVariants[best].items_per_cta;
  TRY(batch_items(b));
  batch_drop_graph(b);
  if (choice) *choice = best;
  return KTUNE_OK;
}

}  // extern "C"
