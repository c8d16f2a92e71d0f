// Reference simulator for the register-level sparse quantum state of SparQSim
// (arXiv 2503.15118).  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and
// the CPU-baseline leg of the benchmark load this file's library; the product
// path never does.
//
// It is deliberately plain and slow: the state is a std::map from the packed
// basis key to a complex<double> amplitude, every operation walks the map once
// and writes a new map, and every number is FP64.  It shares no code, header,
// table or constant with the CUDA library.
//
// Conventions, each taken from the paper and listed with its reading:
//  * State (Sec. II.C, Eq. 5): psi = sum_i a_i |v_i^0>|v_i^1>...|v_i^{K-1}>.
//    Only branches with a nonzero amplitude are stored.
//  * Packing (Sec. II.A, Eq. 4 and Sec. II.C): register j occupies key bits
//    [off_j, off_j + w_j) with off_0 = 0 and off_j = sum_{i<j} w_i, so register 0
//    sits in the low bits and the global qubit index equals the key bit index.
//    Keys are up to 128 bits wide; a register is at most 64 bits wide, the size
//    of one StateStorage value (Table S2).
//  * Controls (Sec. II.A, CU = |0><0| (x) I + |1><1| (x) U; Sec. II.D.1): an
//    operation acts on a branch iff every control bit holds its required value
//    (1 for the textbook control; 0 is accepted as an extension).  Other
//    branches pass through unchanged.
//  * Single-qubit operation U on qubit t (Sec. II.D.2 and the rotation listing
//    of Supp. B): psi'(x) = sum_s U[x_t][s] psi(x with bit t := s); U is indexed
//    [row = output bit][column = input bit], acting on (a0, a1)^T as in Eq. 3.
//    The interference family always ends with the removal of branches whose
//    modulus is below the threshold (ClearZero in Supp. B), whatever the form of
//    U (diagonal, anti-diagonal or general).
//  * Non-interference operations (Sec. II.D.1) -- bit flips under controls,
//    modular arithmetic, register swaps, QRAM and phases -- never remove a branch.
//  * QRAM (Supp. C, Eq. S1): |i>_A |j>_D -> |i>_A |j XOR d_i>_D with d_i taken to
//    the data register's word length.  Addresses past the end of the table read
//    d = 0 (the paper is silent; this keeps the map a bijection).
//  * Pruning (Sec. II.D.2, last paragraph): drop a branch when |a| < eps, strict.
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>

typedef unsigned __int128 u128;
typedef std::complex<double> cplx;

struct OCtrl {
  uint32_t reg, bit, value;
};

struct OState {
  std::vector<uint32_t> width;
  std::vector<uint32_t> offset;
  uint32_t total_bits = 0;
  double eps = 1e-14;
  uint64_t peak = 0;
  std::map<u128, cplx> psi;
};

static u128 low_mask(uint32_t w) {
  if (w >= 128) return ~(u128)0;
  return (((u128)1) << w) - 1;
}

static uint64_t get_reg(const OState* s, u128 key, uint32_t reg) {
  return (uint64_t)((key >> s->offset[reg]) & low_mask(s->width[reg]));
}

static u128 set_reg(const OState* s, u128 key, uint32_t reg, uint64_t value) {
  u128 m = low_mask(s->width[reg]) << s->offset[reg];
  u128 v = (((u128)value) & low_mask(s->width[reg])) << s->offset[reg];
  return (key & ~m) | v;
}

static uint32_t get_bit(const OState* s, u128 key, uint32_t reg, uint32_t bit) {
  return (uint32_t)((key >> (s->offset[reg] + bit)) & 1u);
}

static bool controls_hold(const OState* s, u128 key, const OCtrl* c, uint32_t n) {
  for (uint32_t i = 0; i < n; ++i)
    if (get_bit(s, key, c[i].reg, c[i].bit) != c[i].value) return false;
  return true;
}

static void track_peak(OState* s) {
  if (s->psi.size() > s->peak) s->peak = s->psi.size();
}

static void prune_map(std::map<u128, cplx>& m, double eps) {
  for (auto it = m.begin(); it != m.end();) {
    if (std::abs(it->second) < eps)
      it = m.erase(it);
    else
      ++it;
  }
}

// Applies a key permutation pi to every branch: psi'(pi(k)) = psi(k).
template <class F>
static void permute(OState* s, F pi) {
  std::map<u128, cplx> out;
  for (const auto& kv : s->psi) out[pi(kv.first)] += kv.second;
  s->psi.swap(out);
}

extern "C" {

OState* or_create(const uint32_t* widths, uint32_t n_regs) {
  OState* s = new OState();
  uint32_t off = 0;
  for (uint32_t j = 0; j < n_regs; ++j) {
    s->width.push_back(widths[j]);
    s->offset.push_back(off);
    off += widths[j];
  }
  s->total_bits = off;
  s->psi[(u128)0] = cplx(1.0, 0.0);
  s->peak = 1;
  return s;
}

OState* or_clone(const OState* s) { return new OState(*s); }

void or_destroy(OState* s) { delete s; }

void or_set_eps(OState* s, double eps) { s->eps = eps; }

uint64_t or_nnz(const OState* s) { return (uint64_t)s->psi.size(); }

uint64_t or_peak(const OState* s) { return s->peak; }

// psi'(x) = sum_s U[x_t][s] psi(x with bit t := s) on controlled branches,
// written as a scatter over the stored branches, then pruning.
// m = {re00, im00, re01, im01, re10, im10, re11, im11}.
void or_apply_u1q(OState* s, uint32_t reg, uint32_t bit, const double* m,
                  const OCtrl* ctrl, uint32_t n_ctrl) {
  cplx U[2][2] = {{cplx(m[0], m[1]), cplx(m[2], m[3])},
                  {cplx(m[4], m[5]), cplx(m[6], m[7])}};
  const u128 b = ((u128)1) << (s->offset[reg] + bit);
  std::map<u128, cplx> out;
  for (const auto& kv : s->psi) {
    const u128 k = kv.first;
    const cplx a = kv.second;
    if (!controls_hold(s, k, ctrl, n_ctrl)) {
      out[k] += a;
      continue;
    }
    const uint32_t kt = (k & b) ? 1u : 0u;
    out[k & ~b] += U[0][kt] * a;
    out[k | b] += U[1][kt] * a;
  }
  prune_map(out, s->eps);
  s->psi.swap(out);
  track_peak(s);
}

// H = 2^{-1/2} [[1, 1], [1, -1]] (Sec. II.A).
void or_apply_h(OState* s, uint32_t reg, uint32_t bit, const OCtrl* ctrl, uint32_t n_ctrl) {
  const double r = 1.0 / std::sqrt(2.0);
  const double m[8] = {r, 0, r, 0, r, 0, -r, 0};
  or_apply_u1q(s, reg, bit, m, ctrl, n_ctrl);
}

// RY(theta) = [[cos(theta/2), -sin(theta/2)], [sin(theta/2), cos(theta/2)]]
// (standard convention; the paper names rotations without fixing one).
void or_apply_ry(OState* s, uint32_t reg, uint32_t bit, double theta, const OCtrl* ctrl,
                 uint32_t n_ctrl) {
  const double c = std::cos(theta / 2), sn = std::sin(theta / 2);
  const double m[8] = {c, 0, -sn, 0, sn, 0, c, 0};
  or_apply_u1q(s, reg, bit, m, ctrl, n_ctrl);
}

// Register-valued rotation (the angle_function_t of the rotation listing in
// Supp. B): the 2x2 applied to a branch is RY(angle) with
// angle = scale * value(angle_reg) + offset, the angle register read from the
// branch itself.  The angle register must not contain the target qubit.
void or_apply_ry_reg(OState* s, uint32_t reg, uint32_t bit, uint32_t angle_reg, double scale,
                     double offset, const OCtrl* ctrl, uint32_t n_ctrl) {
  const u128 b = ((u128)1) << (s->offset[reg] + bit);
  std::map<u128, cplx> out;
  for (const auto& kv : s->psi) {
    const u128 k = kv.first;
    const cplx a = kv.second;
    if (!controls_hold(s, k, ctrl, n_ctrl)) {
      out[k] += a;
      continue;
    }
    const double theta = scale * (double)get_reg(s, k, angle_reg) + offset;
    const double c = std::cos(theta / 2), sn = std::sin(theta / 2);
    const cplx U[2][2] = {{cplx(c, 0), cplx(-sn, 0)}, {cplx(sn, 0), cplx(c, 0)}};
    const uint32_t kt = (k & b) ? 1u : 0u;
    out[k & ~b] += U[0][kt] * a;
    out[k | b] += U[1][kt] * a;
  }
  prune_map(out, s->eps);
  s->psi.swap(out);
  track_peak(s);
}

// X under controls: flip bit t (FlipBool in Supp. B; CNOT / Toffoli with controls).
void or_apply_x(OState* s, uint32_t reg, uint32_t bit, const OCtrl* ctrl, uint32_t n_ctrl) {
  const u128 b = ((u128)1) << (s->offset[reg] + bit);
  permute(s, [&](u128 k) { return controls_hold(s, k, ctrl, n_ctrl) ? (k ^ b) : k; });
}

// Modular adder (quantum arithmetic, Sec. II.D.1):
// dst := (dst + src) mod 2^{w_dst}, or (dst - src) when subtract != 0.
// src is register src_reg, or the constant when src_reg < 0.
void or_apply_add(OState* s, uint32_t dst, int32_t src_reg, uint64_t constant, int32_t subtract,
                  const OCtrl* ctrl, uint32_t n_ctrl) {
  const uint32_t w = s->width[dst];
  const u128 mod_mask = low_mask(w);
  permute(s, [&](u128 k) {
    if (!controls_hold(s, k, ctrl, n_ctrl)) return k;
    const u128 d = get_reg(s, k, dst);
    const u128 v = (src_reg >= 0) ? (u128)get_reg(s, k, (uint32_t)src_reg) : (u128)constant;
    // Arithmetic wraps modulo 2^128, a multiple of 2^w, then is reduced modulo 2^w.
    const u128 r = subtract ? ((d - v) & mod_mask) : ((d + v) & mod_mask);
    return set_reg(s, k, dst, (uint64_t)r);
  });
}

// The arithmetic oracles of Sec. II.D.1 in reversible form: multiply-add
// dst := (dst + a b) mod 2^w, multiply by an odd constant dst := (dst c) mod
// 2^w, and divide-XOR dst := dst XOR floor(a / b) (0 when b = 0).
void or_apply_mul_add(OState* s, uint32_t dst, uint32_t src1, uint32_t src2, const OCtrl* ctrl,
                      uint32_t n_ctrl) {
  const u128 m = low_mask(s->width[dst]);
  permute(s, [&](u128 k) {
    if (!controls_hold(s, k, ctrl, n_ctrl)) return k;
    const u128 d = get_reg(s, k, dst);
    const u128 a = get_reg(s, k, src1), b = get_reg(s, k, src2);
    return set_reg(s, k, dst, (uint64_t)((d + a * b) & m));
  });
}

void or_apply_mul_const(OState* s, uint32_t dst, uint64_t c, const OCtrl* ctrl, uint32_t n_ctrl) {
  const u128 m = low_mask(s->width[dst]);
  permute(s, [&](u128 k) {
    if (!controls_hold(s, k, ctrl, n_ctrl)) return k;
    const u128 d = get_reg(s, k, dst);
    return set_reg(s, k, dst, (uint64_t)((d * (u128)c) & m));
  });
}

void or_apply_div_xor(OState* s, uint32_t dst, uint32_t src1, uint32_t src2, const OCtrl* ctrl,
                      uint32_t n_ctrl) {
  const u128 m = low_mask(s->width[dst]);
  permute(s, [&](u128 k) {
    if (!controls_hold(s, k, ctrl, n_ctrl)) return k;
    const uint64_t a = get_reg(s, k, src1), b = get_reg(s, k, src2);
    const uint64_t q = b ? a / b : 0;
    return set_reg(s, k, dst, (uint64_t)(((u128)get_reg(s, k, dst) ^ (u128)q) & m));
  });
}

// Exchange of two registers of equal width.
void or_apply_swap(OState* s, uint32_t r1, uint32_t r2, const OCtrl* ctrl, uint32_t n_ctrl) {
  permute(s, [&](u128 k) {
    if (!controls_hold(s, k, ctrl, n_ctrl)) return k;
    const uint64_t v1 = get_reg(s, k, r1), v2 = get_reg(s, k, r2);
    return set_reg(s, set_reg(s, k, r1, v2), r2, v1);
  });
}

// Diagonal phase: a := a * e^{i phi} on every branch where all predicates hold
// (Z, S, T and their controlled forms, Sec. II.D.1).
void or_apply_phase(OState* s, const OCtrl* pred, uint32_t n_pred, double phi) {
  const cplx f = std::polar(1.0, phi);
  for (auto& kv : s->psi)
    if (controls_hold(s, kv.first, pred, n_pred)) kv.second *= f;
}

// QRAM load (Supp. C, Eq. S1): data := data XOR d_addr, d truncated to the
// data register's word length.  The same map undoes itself, so unload calls
// this function again.
// The address is the concatenation of registers addr_reg .. addr_reg +
// n_addr - 1, register addr_reg lowest (one register when n_addr = 1).
void or_qram_span(OState* s, uint32_t addr_reg, uint32_t n_addr, uint32_t data_reg,
                  const void* table, uint64_t n_entries, uint32_t entry_bytes) {
  const uint64_t wmask = (uint64_t)low_mask(s->width[data_reg]);
  permute(s, [&](u128 k) {
    uint64_t i = 0;
    uint32_t shift = 0;
    for (uint32_t r = addr_reg; r < addr_reg + n_addr; ++r) {
      i |= get_reg(s, k, r) << shift;
      shift += s->width[r];
    }
    uint64_t d = 0;
    if (i < n_entries) {
      const unsigned char* p = (const unsigned char*)table + i * entry_bytes;
      // Little-endian read of one entry.
      for (uint32_t byte = 0; byte < entry_bytes; ++byte) d |= ((uint64_t)p[byte]) << (8 * byte);
    }
    return set_reg(s, k, data_reg, get_reg(s, k, data_reg) ^ (d & wmask));
  });
}

void or_qram(OState* s, uint32_t addr_reg, uint32_t data_reg, const void* table,
             uint64_t n_entries, uint32_t entry_bytes) {
  or_qram_span(s, addr_reg, 1, data_reg, table, n_entries, entry_bytes);
}

void or_prune(OState* s, double eps) { prune_map(s->psi, eps); }

// Writes the branches in ascending key order: keys as (lo, hi) pairs of
// 64-bit words, amplitudes as (re, im).  Returns the number written.
uint64_t or_export(const OState* s, uint64_t* keys_lo, uint64_t* keys_hi, double* amps,
                   uint64_t cap) {
  uint64_t n = 0;
  for (const auto& kv : s->psi) {
    if (n >= cap) break;
    keys_lo[n] = (uint64_t)kv.first;
    keys_hi[n] = (uint64_t)(kv.first >> 64);
    amps[2 * n] = kv.second.real();
    amps[2 * n + 1] = kv.second.imag();
    ++n;
  }
  return n;
}

// Replaces the state with the given branches (keys must be distinct).
void or_import(OState* s, const uint64_t* keys_lo, const uint64_t* keys_hi, const double* amps,
               uint64_t n) {
  s->psi.clear();
  for (uint64_t i = 0; i < n; ++i) {
    u128 k = (((u128)keys_hi[i]) << 64) | keys_lo[i];
    s->psi[k] += cplx(amps[2 * i], amps[2 * i + 1]);
  }
  track_peak(s);
}

// Marginal probabilities of one register: p(v) = sum_{k: reg(k) = v} |a_k|^2,
// written for the distinct values in ascending order.  Returns the count.
uint64_t or_probabilities(const OState* s, uint32_t reg, uint64_t* values, double* probs,
                          uint64_t cap) {
  std::map<uint64_t, double> p;
  for (const auto& kv : s->psi) p[get_reg(s, kv.first, reg)] += std::norm(kv.second);
  uint64_t n = 0;
  for (const auto& kv : p) {
    if (n >= cap) break;
    values[n] = kv.first;
    probs[n] = kv.second;
    ++n;
  }
  return n;
}

// Squared norm, sum_k |a_k|^2.
double or_norm2(const OState* s) {
  double t = 0;
  for (const auto& kv : s->psi) t += std::norm(kv.second);
  return t;
}

// Amplitude of one key (0 when absent).
void or_amplitude(const OState* s, uint64_t key_lo, uint64_t key_hi, double* re, double* im) {
  u128 k = (((u128)key_hi) << 64) | key_lo;
  auto it = s->psi.find(k);
  *re = (it == s->psi.end()) ? 0.0 : it->second.real();
  *im = (it == s->psi.end()) ? 0.0 : it->second.imag();
}

}  // extern "C"
