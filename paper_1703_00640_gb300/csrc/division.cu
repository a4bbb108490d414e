// Division built on the truncated products: the reciprocal of a k-bit divisor by
// Newton's iteration (high and low products of growing size) and Barrett's
// quotient (one high and one low product per division). Section 1 of the paper
// names Barrett's reduction as an application of the high product. The limb
// arithmetic between the products (shifts, additions with carry propagation,
// sign tests, small corrections) runs in the kernels of this file.
#include <algorithm>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/truncmul.h"
#include "runtime.h"

namespace tmul {
namespace {

using u64 = unsigned long long;

// ------------------------------------------------------------ limb kernels

constexpr int kLopThreads = 256;
constexpr int kLopPer = 8;
constexpr long long kLopTile = kLopThreads * kLopPer;   // limbs per block
constexpr int kScanThreads = 1024;

// Carry behaviour of a run of limbs: carry out = g | (p & carry in).
struct GP {
  unsigned g, p;
};
__device__ __forceinline__ GP gp_compose(GP lo, GP hi) { return {hi.g | (hi.p & lo.g), hi.p & lo.p}; }

enum { kCondAlways = 0, kCondFlag, kCondANeg, kCondBNeg, kCondResultNonneg };

// out = a + b' + cin mod 2^(64 W), b' = ~b and cin = 1 when negating (a - b), else
// b' = b and cin = 0. a, b are zero-extended beyond na, nb limbs (nullptr = 0);
// b_small replaces b by the sign-extended value *b_small. Signs are those of
// W-limb two's complement values. The sum is written only when the condition
// holds; otherwise out receives keep (nullptr: a).
struct LopArgs {
  const u64* a;
  long long na;
  const u64* b;
  long long nb;
  const long long* b_small;
  u64* out;
  long long W;
  const u64* keep;
  long long nkeep;
  int negate;                  // 0, 1, or -1: read *neg_flag
  const int* neg_flag;
  int cond;
  const int* cond_flag;
  int* applied_out;            // nullable: 1 when the sum was written
  long long* delta;            // nullable: *delta += dinc when the sum was written
  int dinc;
  GP* blk;                     // scratch: per-block carry behaviour
  unsigned* bcin;              // scratch: per-block carry in
  int* applied;                // scratch: condition, read by the apply kernel
};

__device__ __forceinline__ u64 limb_at(const u64* x, long long n, long long i) {
  return (x && i < n) ? x[i] : 0ull;
}

__device__ __forceinline__ bool neg_of(const LopArgs& a) {
  return a.negate < 0 ? (*a.neg_flag != 0) : (a.negate != 0);
}

__device__ __forceinline__ u64 b_at(const LopArgs& a, long long i, bool neg) {
  u64 y;
  if (a.b_small) {
    const long long v = *a.b_small;
    y = i == 0 ? (u64)v : (v < 0 ? ~0ull : 0ull);
  } else {
    y = limb_at(a.b, a.nb, i);
  }
  return neg ? ~y : y;
}

// Exclusive scan of carry behaviours over the block (thread order); *total gets
// the composition over all threads. Every thread of the block must call it.
template <int NT>
__device__ GP block_exclusive(GP x, GP* total) {
  __shared__ GP wsum[NT / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  GP inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned g = __shfl_up_sync(~0u, inc.g, o), p = __shfl_up_sync(~0u, inc.p, o);
    if (lane >= o) inc = gp_compose(GP{g, p}, inc);
  }
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    GP w = lane < NT / 32 ? wsum[lane] : GP{0u, 1u};
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned g = __shfl_up_sync(~0u, w.g, o), p = __shfl_up_sync(~0u, w.p, o);
      if (lane >= o) w = gp_compose(GP{g, p}, w);
    }
    if (lane < NT / 32) wsum[lane] = w;
  }
  __syncthreads();
  const unsigned g1 = __shfl_up_sync(~0u, inc.g, 1), p1 = __shfl_up_sync(~0u, inc.p, 1);
  const GP ex_lane = lane == 0 ? GP{0u, 1u} : GP{g1, p1};
  const GP before = wid == 0 ? GP{0u, 1u} : wsum[wid - 1];
  const GP ex = gp_compose(before, ex_lane);
  if (total) *total = wsum[NT / 32 - 1];
  __syncthreads();
  return ex;
}

__device__ __forceinline__ GP limb_gp(u64 x, u64 y) {
  const u64 s = x + y;
  return GP{s < x ? 1u : 0u, s == ~0ull ? 1u : 0u};
}

// 1. carry behaviour of each block's limbs
__global__ void __launch_bounds__(kLopThreads) k_lop_local(LopArgs a) {
  pdl_trigger();
  pdl_wait();
  const bool neg = neg_of(a);
  const long long base = blockIdx.x * kLopTile + (long long)threadIdx.x * kLopPer;
  GP t{0u, 1u};
  for (int i = 0; i < kLopPer; ++i) {
    const long long idx = base + i;
    if (idx >= a.W) break;
    t = gp_compose(t, limb_gp(limb_at(a.a, a.na, idx), b_at(a, idx, neg)));
  }
  GP total;
  block_exclusive<kLopThreads>(t, &total);
  if (threadIdx.x == 0) a.blk[blockIdx.x] = total;
}

// 2. carry into every block (one CTA), the top limb's value and the condition
__global__ void __launch_bounds__(kScanThreads) k_lop_scan(LopArgs a, long long nblk) {
  pdl_trigger();
  pdl_wait();
  const bool neg = neg_of(a);
  const unsigned cin0 = neg ? 1u : 0u;
  const long long per = (nblk + kScanThreads - 1) / kScanThreads;
  const long long j0 = threadIdx.x * per, j1 = j0 + per < nblk ? j0 + per : nblk;
  GP t{0u, 1u};
  for (long long j = j0; j < j1; ++j) t = gp_compose(t, a.blk[j]);
  const GP ex = block_exclusive<kScanThreads>(t, nullptr);
  unsigned c = ex.g | (ex.p & cin0);
  __shared__ unsigned ctop;
  for (long long j = j0; j < j1; ++j) {
    a.bcin[j] = c;
    if (j == nblk - 1) ctop = c;
    const GP x = a.blk[j];
    c = x.g | (x.p & c);
  }
  __syncthreads();
  // carry into limb W-1: the top block's limbs below it, two per thread
  const long long tb = (nblk - 1) * kLopTile;
  GP s{0u, 1u};
  for (int i = 0; i < 2; ++i) {
    const long long idx = tb + 2LL * threadIdx.x + i;
    if (idx < a.W - 1) s = gp_compose(s, limb_gp(limb_at(a.a, a.na, idx), b_at(a, idx, neg)));
  }
  GP tot;
  block_exclusive<kScanThreads>(s, &tot);
  if (threadIdx.x == 0) {
    const long long ti = a.W - 1;
    const unsigned cin_top = tot.g | (tot.p & ctop);
    const u64 at = limb_at(a.a, a.na, ti);
    const u64 rt = at + b_at(a, ti, neg) + cin_top;
    bool ap;
    switch (a.cond) {
      case kCondAlways: ap = true; break;
      case kCondFlag: ap = *a.cond_flag != 0; break;
      case kCondANeg: ap = (at >> 63) != 0; break;
      case kCondBNeg: ap = a.b_small ? (*a.b_small < 0) : ((limb_at(a.b, a.nb, ti) >> 63) != 0); break;
      case kCondResultNonneg: ap = (rt >> 63) == 0; break;
      default: ap = false;
    }
    *a.applied = ap ? 1 : 0;
    if (a.applied_out) *a.applied_out = ap ? 1 : 0;
    if (a.delta && ap) *a.delta += a.dinc;
  }
}

// 3. the limbs of the sum (or of keep)
__global__ void __launch_bounds__(kLopThreads) k_lop_apply(LopArgs a) {
  pdl_trigger();
  pdl_wait();
  const bool neg = neg_of(a);
  const bool ap = *a.applied != 0;
  const long long base = blockIdx.x * kLopTile + (long long)threadIdx.x * kLopPer;
  u64 s[kLopPer];
  unsigned gb = 0, pb = 0;
  GP t{0u, 1u};
#pragma unroll
  for (int i = 0; i < kLopPer; ++i) {
    const long long idx = base + i;
    s[i] = 0;
    if (idx < a.W) {
      const u64 x = limb_at(a.a, a.na, idx);
      s[i] = x + b_at(a, idx, neg);
      const GP q{s[i] < x ? 1u : 0u, s[i] == ~0ull ? 1u : 0u};
      gb |= q.g << i;
      pb |= q.p << i;
      t = gp_compose(t, q);
    }
  }
  const GP ex = block_exclusive<kLopThreads>(t, nullptr);
  unsigned c = ex.g | (ex.p & a.bcin[blockIdx.x]);
  const u64* keep = a.keep ? a.keep : a.a;
  const long long nkeep = a.keep ? a.nkeep : a.na;
#pragma unroll
  for (int i = 0; i < kLopPer; ++i) {
    const long long idx = base + i;
    if (idx >= a.W) break;
    if (ap) {
      a.out[idx] = s[i] + c;
    } else if (keep != a.out) {
      a.out[idx] = limb_at(keep, nkeep, idx);
    }
    c = ((gb >> i) & 1u) | (((pb >> i) & 1u) & c);
  }
}

// 64 bits of the src_bits-bit integer src starting at bit pos (zero outside
// [0, src_bits); pos may be negative).
__device__ __forceinline__ u64 field64(const u64* src, long long ns, long long src_bits,
                                       long long pos) {
  if (pos >= src_bits || pos <= -64) return 0ull;
  const long long q = pos >= 0 ? pos / 64 : -((-pos + 63) / 64);
  const int sh = int(pos - 64 * q);
  const u64 l0 = (q >= 0 && q < ns) ? src[q] : 0ull;
  const u64 l1 = (q + 1 >= 0 && q + 1 < ns) ? src[q + 1] : 0ull;
  u64 r = sh ? ((l0 >> sh) | (l1 << (64 - sh))) : l0;
  const long long valid = src_bits - pos;
  if (valid < 64) r &= (1ull << valid) - 1ull;
  return r;
}

// dst[i] = bits [64 i + off, 64 i + off + 64) of src, complemented when invert, cut
// to dst_bits bits; i < nd. dst must not overlap src.
__global__ void k_bits(u64* dst, long long nd, long long dst_bits, const u64* src, long long ns,
                       long long src_bits, long long off, int invert) {
  pdl_trigger();
  pdl_wait();
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nd) return;
  u64 x = field64(src, ns, src_bits, 64 * i + off);
  if (invert) x = ~x;
  const long long lo = 64 * i;
  if (dst_bits <= lo) x = 0;
  else if (dst_bits < lo + 64) x &= (1ull << (dst_bits - lo)) - 1ull;
  dst[i] = x;
}

// v (W limbs) := the p-bit two's complement value in its low p bits, sign-extended.
__global__ void k_sext(u64* v, long long W, long long p) {
  pdl_trigger();
  pdl_wait();
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= W) return;
  const bool sign = (v[(p - 1) / 64] >> ((p - 1) % 64)) & 1ull;   // bit p-1 is never rewritten
  const long long lo = 64 * i;
  if (lo + 64 <= p) return;
  const u64 fill = sign ? ~0ull : 0ull;
  if (lo >= p) {
    v[i] = fill;
  } else {
    const u64 keep = (1ull << (p - lo)) - 1ull;
    v[i] = (v[i] & keep) | (fill & ~keep);
  }
}

// X = floor((2^(2h) - 1) / m_h), m_h = bits [k-h, k) of m, h <= 60: binary long
// division on one thread (every bit of the dividend is one).
__global__ void k_recip_base(u64* X, long long nX, const u64* m, long long nm, long long k,
                             int h) {
  pdl_trigger();
  pdl_wait();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const u64 mh = field64(m, nm, k, k - h) & ((1ull << h) - 1ull);
  u64 rem = 0, q = 0;
  for (int i = 0; i < 2 * h; ++i) {
    rem = 2 * rem + 1;
    q *= 2;
    if (rem >= mh) {
      rem -= mh;
      q += 1;
    }
  }
  X[0] = q;
  for (long long i = 1; i < nX; ++i) X[i] = 0;
}

// ------------------------------------------------------------ host side

int64_t L(int64_t bits) { return (bits + 63) / 64; }

int cuda_rc(cudaError_t e) {
  if (e == cudaSuccess) return TM_OK;
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? TM_ENOMEM : TM_ECUDA;
}

// Device flags of one division context.
struct Flags {
  long long delta;             // quotient (or reciprocal) correction
  long long fail;              // final range checks that did not hold
  int sign;                    // sign of E in the current Newton step
  int pad[3];
};

// Scratch and launchers for the limb kernels on one stream.
struct Limbs {
  cudaStream_t s = nullptr;
  char* mem = nullptr;
  GP* blk = nullptr;
  unsigned* bcin = nullptr;
  int* applied = nullptr;
  Flags* flags = nullptr;
  long long max_blocks = 0;

  int init(long long max_limbs, cudaStream_t st) {
    s = st;
    max_blocks = (max_limbs + kLopTile - 1) / kLopTile + 1;
    const size_t bytes = align_up(max_blocks * sizeof(GP)) + align_up(max_blocks * 4) + 256 +
                         align_up(sizeof(Flags));
    int rc = cuda_rc(cudaMalloc(&mem, bytes));
    if (rc) return rc;
    blk = reinterpret_cast<GP*>(mem);
    bcin = reinterpret_cast<unsigned*>(mem + align_up(max_blocks * sizeof(GP)));
    applied = reinterpret_cast<int*>(mem + align_up(max_blocks * sizeof(GP)) +
                                     align_up(max_blocks * 4));
    flags = reinterpret_cast<Flags*>(reinterpret_cast<char*>(applied) + 256);
    return cuda_rc(cudaMemsetAsync(flags, 0, sizeof(Flags), s));
  }
  void release() {
    if (mem) cudaFree(mem);
    mem = nullptr;
  }
  void bits(u64* dst, long long nd, long long dst_bits, const u64* src, long long ns,
            long long src_bits, long long off, bool invert = false) const {
    const unsigned grid = unsigned((nd + 255) / 256);
    launch_pdl(k_bits, dim3(grid), dim3(256), 0, s, dst, nd, dst_bits, src, ns, src_bits, off,
               invert ? 1 : 0);
  }
  void sext(u64* v, long long W, long long p) const {
    launch_pdl(k_sext, dim3(unsigned((W + 255) / 256)), dim3(256), 0, s, v, W, p);
  }
  void lop(LopArgs a) const {
    const long long nblk = (a.W + kLopTile - 1) / kLopTile;
    a.blk = blk;
    a.bcin = bcin;
    a.applied = applied;
    launch_pdl(k_lop_local, dim3(unsigned(nblk)), dim3(kLopThreads), 0, s, a);
    launch_pdl(k_lop_scan, dim3(1), dim3(kScanThreads), 0, s, a, nblk);
    launch_pdl(k_lop_apply, dim3(unsigned(nblk)), dim3(kLopThreads), 0, s, a);
  }
};

LopArgs sum(u64* out, long long W, const u64* a, long long na, const u64* b, long long nb,
            bool negate) {
  LopArgs x{};
  x.a = a; x.na = na; x.b = b; x.nb = nb; x.out = out; x.W = W;
  x.negate = negate ? 1 : 0;
  x.cond = kCondAlways;
  return x;
}

// A device buffer of limbs owned by the caller of alloc_limbs.
int alloc_limbs(u64** p, long long n) {
  return cuda_rc(cudaMalloc(p, size_t(std::max<long long>(n, 1)) * 8));
}

// Checks that bit k-1 of m is set (the divisor has exactly k bits).
int check_top_bit(const u64* m, uint64_t k, cudaStream_t s) {
  u64 top = 0;
  int rc = cuda_rc(cudaMemcpyAsync(&top, m + (k - 1) / 64, 8, cudaMemcpyDeviceToHost, s));
  if (rc) return rc;
  rc = cuda_rc(cudaStreamSynchronize(s));
  if (rc) return rc;
  return ((top >> ((k - 1) % 64)) & 1ull) ? TM_OK : TM_EINVAL;
}

// R = floor((2^(2k) - 1) / m) into R (L(k+1) limbs), m with bit k-1 set; enqueued on
// lm.s; scratch buffers sized for k.
int reciprocal(u64* R, const u64* m, int64_t k, Limbs& lm) {
  cudaStream_t s = lm.s;
  if (k <= 60) {
    u64* X = nullptr;
    int rc = alloc_limbs(&X, 2);
    if (rc) return rc;
    k_recip_base<<<1, 32, 0, s>>>(X, 2, m, L(k), k, int(k));
    lm.bits(R, L(k + 1), k + 1, X, 2, 128, 0);
    rc = cuda_rc(cudaStreamSynchronize(s));
    cudaFree(X);
    return rc;
  }
  // precisions k = H_t > ... > H_0 <= 60 with 2 H_i >= H_(i+1) + 9
  std::vector<int64_t> hs{k};
  while (hs.back() > 60) hs.push_back(hs.back() / 2 + 5);
  const int64_t S = L(k + 16) + 2;
  std::vector<u64*> buf(12, nullptr);
  for (auto& p : buf) {
    int rc = alloc_limbs(&p, S);
    if (rc) {
      for (auto q : buf) if (q) cudaFree(q);
      return rc;
    }
  }
  u64 *X = buf[0], *Y = buf[1], *mH = buf[2], *Xz = buf[3], *lo = buf[4], *E = buf[5],
      *absE = buf[6], *Xh = buf[7], *Eh = buf[8], *corr = buf[9], *Xs = buf[10], *e = buf[11];
  int64_t h = hs.back(), nX = 2;
  k_recip_base<<<1, 32, 0, s>>>(X, nX, m, L(k), k, int(h));
  int rc = TM_OK;
  for (int li = int(hs.size()) - 2; li >= 0 && rc == TM_OK; --li) {
    // Newton step from precision h to H: Y = X 2^(H-h) + X E' / 2^(2h),
    // E' = 2^(H+h) - m_H X (|E'| < 2^(H+4), from a low product mod 2^(H+5))
    const int64_t H = hs[li];
    const int64_t n5 = L(H + 5), WE = n5 + 1;
    lm.bits(mH, n5, H, m, L(k), k, k - H);
    lm.bits(Xz, n5, h + 2, X, nX, h + 2, 0);
    rc = tm_mul(TM_LO, reinterpret_cast<uint64_t*>(lo), reinterpret_cast<uint64_t*>(mH),
                reinterpret_cast<uint64_t*>(Xz), uint64_t(H + 5), s, nullptr);
    if (rc) break;
    lm.lop(sum(E, WE, nullptr, 0, lo, n5, true));
    lm.sext(E, WE, H + 5);
    LopArgs ab = sum(absE, WE, nullptr, 0, E, WE, true);    // |E'|; flags.sign = [E' < 0]
    ab.cond = kCondBNeg;
    ab.keep = E;
    ab.nkeep = WE;
    ab.applied_out = &lm.flags->sign;
    lm.lop(ab);
    const int64_t n2h = L(2 * h);
    lm.bits(Xh, n2h, 2 * h, X, nX, h + 2, 0);
    lm.bits(Eh, n2h, 2 * h, absE, WE, 64 * WE, 0);
    rc = tm_mul(TM_HI, reinterpret_cast<uint64_t*>(corr), reinterpret_cast<uint64_t*>(Xh),
                reinterpret_cast<uint64_t*>(Eh), uint64_t(2 * h), s, nullptr);
    if (rc) break;
    const int64_t WY = L(H + 2) + 1;
    lm.bits(Xs, WY, H + 2, X, nX, h + 2, -(H - h));
    LopArgs y = sum(Y, WY, Xs, WY, corr, (2 * h) / 64 + 1, false);
    y.negate = -1;
    y.neg_flag = &lm.flags->sign;
    lm.lop(y);
    std::swap(X, Y);
    nX = WY;
    h = H;
  }
  if (rc == TM_OK) {
    // exact correction: e = 2^(2k) - 1 - m X (mod 2^(k+4), signed), then
    // X += floor(e / m) by single steps (|X - R| <= 4)
    const int64_t n4 = L(k + 4), We = n4 + 1;
    lm.bits(mH, n4, k, m, L(k), k, 0);
    lm.bits(Xz, n4, k + 2, X, nX, k + 2, 0);
    rc = tm_mul(TM_LO, reinterpret_cast<uint64_t*>(lo), reinterpret_cast<uint64_t*>(mH),
                reinterpret_cast<uint64_t*>(Xz), uint64_t(k + 4), s, nullptr);
    if (rc == TM_OK) {
      lm.bits(e, We, k + 4, lo, n4, k + 4, 0, true);
      lm.sext(e, We, k + 4);
      for (int i = 0; i < 6; ++i) {                 // e < 0: e += m, X -= 1
        LopArgs a = sum(e, We, e, We, mH, n4, false);
        a.cond = kCondANeg;
        a.delta = &lm.flags->delta;
        a.dinc = -1;
        lm.lop(a);
      }
      for (int i = 0; i < 6; ++i) {                 // e >= m: e -= m, X += 1
        LopArgs a = sum(e, We, e, We, mH, n4, true);
        a.cond = kCondResultNonneg;
        a.delta = &lm.flags->delta;
        a.dinc = 1;
        lm.lop(a);
      }
      for (int neg = 0; neg < 2; ++neg) {           // 0 <= e < m must hold now
        LopArgs a = sum(e, We, e, We, mH, n4, neg == 1);
        a.cond = neg ? kCondResultNonneg : kCondANeg;
        a.delta = &lm.flags->fail;
        a.dinc = 1;
        lm.lop(a);
      }
      LopArgs f{};
      f.a = X; f.na = nX; f.b_small = &lm.flags->delta; f.out = Y; f.W = nX;
      f.cond = kCondAlways;
      lm.lop(f);
      lm.bits(R, L(k + 1), k + 1, Y, nX, 64 * nX, 0);
    }
  }
  if (rc == TM_OK) rc = cuda_rc(cudaGetLastError());
  if (rc == TM_OK) {
    Flags fl{};
    rc = cuda_rc(cudaMemcpyAsync(&fl, lm.flags, sizeof(Flags), cudaMemcpyDeviceToHost, s));
    if (rc == TM_OK) rc = cuda_rc(cudaStreamSynchronize(s));
    if (rc == TM_OK && fl.fail) rc = TM_EPRECISION;
  } else {
    cudaStreamSynchronize(s);
  }
  for (auto p : buf) cudaFree(p);
  return rc;
}

}  // namespace
}  // namespace tmul

// A divisor m of k bits with its reciprocal and the kept transforms of both.
struct tm_barrett {
  uint64_t k;
  int device;
  tmul::u64* R;                // floor((2^(2k) - 1) / m), L(k+1) limbs
  tmul::u64* mW;               // m, L(k+3) + 1 limbs
  tm_operand* opR;             // high product, n = k + 1
  tm_operand* opM;             // low product, n = k + 3
  tmul::u64* x1;               // floor(x / 2^(k-1))
  tmul::u64* qh;               // high product output
  tmul::u64* qz;               // q^ on k + 3 bits
  tmul::u64* t;                // q^ m mod 2^(k+3)
  tmul::u64* xl;               // x mod 2^(k+3)
  tmul::u64* rr;               // remainder window
  tmul::u64* qq;               // corrected quotient
  tm_report plan_hi, plan_lo;  // plans of the two products
  tmul::Limbs lm;
};

namespace {

void barrett_free(tm_barrett* b) {
  if (!b) return;
  if (b->opR) tm_operand_destroy(b->opR);
  if (b->opM) tm_operand_destroy(b->opM);
  for (tmul::u64* p : {b->R, b->mW, b->x1, b->qh, b->qz, b->t, b->xl, b->rr, b->qq})
    if (p) cudaFree(p);
  b->lm.release();
  delete b;
}

int check_k(uint64_t k) {
  if (k == 0) return TM_EINVAL;
  if (k > TM_MAX_BITS - 16) return TM_ERANGE;
  return TM_OK;
}

}  // namespace

extern "C" {

int tm_reciprocal(uint64_t* R, const uint64_t* m, uint64_t k_bits, void* stream) {
  if (!R || !m) return TM_EINVAL;
  int rc = check_k(k_bits);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const tmul::u64* dm = reinterpret_cast<const tmul::u64*>(m);
  rc = tmul::check_top_bit(dm, k_bits, s);
  if (rc) return rc;
  tmul::Limbs lm;
  rc = lm.init(tmul::L(int64_t(k_bits) + 16) + 2, s);
  if (rc == TM_OK) rc = tmul::reciprocal(reinterpret_cast<tmul::u64*>(R), dm, int64_t(k_bits), lm);
  if (rc == TM_OK) {
    tm_report rep{};
    const int st = tm_stream_status(stream, &rep);
    if (st) rc = st;
  }
  lm.release();
  return rc;
}

int tm_barrett_create(const uint64_t* m, uint64_t k_bits, void* stream, tm_barrett** out) {
  if (!out || !m) return TM_EINVAL;
  *out = nullptr;
  int rc = check_k(k_bits);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t k = int64_t(k_bits);
  const tmul::u64* dm = reinterpret_cast<const tmul::u64*>(m);
  rc = tmul::check_top_bit(dm, k_bits, s);
  if (rc) return rc;
  tm_barrett* b = new tm_barrett{};
  b->k = k_bits;
  cudaGetDevice(&b->device);
  const int64_t n3 = tmul::L(k + 3), Wr = n3 + 1;
  rc = b->lm.init(tmul::L(k + 16) + 2, s);           // the Newton steps' widths too
  if (!rc) rc = tmul::alloc_limbs(&b->R, tmul::L(k + 1));
  if (!rc) rc = tmul::alloc_limbs(&b->mW, Wr);
  if (!rc) rc = tmul::alloc_limbs(&b->x1, tmul::L(k + 1));
  if (!rc) rc = tmul::alloc_limbs(&b->qh, (k + 1) / 64 + 1);
  if (!rc) rc = tmul::alloc_limbs(&b->qz, n3);
  if (!rc) rc = tmul::alloc_limbs(&b->t, n3);
  if (!rc) rc = tmul::alloc_limbs(&b->xl, n3);
  if (!rc) rc = tmul::alloc_limbs(&b->rr, Wr);
  if (!rc) rc = tmul::alloc_limbs(&b->qq, Wr);
  if (!rc) rc = tmul::reciprocal(b->R, dm, k, b->lm);
  if (!rc) {
    b->lm.bits(b->mW, Wr, k, dm, tmul::L(k), k, 0);
    rc = tm_operand_create(TM_HI, k_bits + 1, reinterpret_cast<uint64_t*>(b->R), stream, &b->opR);
  }
  if (!rc)
    rc = tm_operand_create(TM_LO, k_bits + 3, reinterpret_cast<uint64_t*>(b->mW), stream,
                           &b->opM);
  if (!rc) rc = tm_plan_query(TM_HI, k_bits + 1, &b->plan_hi);
  if (!rc) rc = tm_plan_query(TM_LO, k_bits + 3, &b->plan_lo);
  if (!rc) rc = tmul::cuda_rc(cudaStreamSynchronize(s));
  if (rc) {
    barrett_free(b);
    return rc;
  }
  *out = b;
  return TM_OK;
}

int tm_barrett_reciprocal(const tm_barrett* b, uint64_t* R, void* stream) {
  if (!b || !R) return TM_EINVAL;
  const size_t bytes = size_t(tmul::L(int64_t(b->k) + 1)) * 8;
  return tmul::cuda_rc(cudaMemcpyAsync(R, b->R, bytes, cudaMemcpyDeviceToDevice,
                                       static_cast<cudaStream_t>(stream)));
}

int tm_barrett_divrem(tm_barrett* b, uint64_t* q, uint64_t* r, const uint64_t* x, void* stream,
                      tm_report* rep) {
  using tmul::u64;
  if (!b || !x || (!q && !r)) return TM_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TM_ECUDA;
  if (dev != b->device) return TM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tmul::Limbs& lm = b->lm;
  lm.s = s;
  const int64_t k = int64_t(b->k), n3 = tmul::L(k + 3), Wr = n3 + 1, nx = tmul::L(2 * k);
  const u64* dx = reinterpret_cast<const u64*>(x);
  int rc = tmul::cuda_rc(cudaMemsetAsync(lm.flags, 0, sizeof(tmul::Flags), s));
  if (rc) return rc;
  // q^ = round(x1 R / 2^(k+1)), x1 = floor(x / 2^(k-1)): q - 3 <= q^ <= q + 1
  lm.bits(b->x1, tmul::L(k + 1), k + 1, dx, nx, 2 * k, k - 1);
  rc = tm_mul_operand(reinterpret_cast<uint64_t*>(b->qh), reinterpret_cast<uint64_t*>(b->x1),
                      b->opR, stream, nullptr);
  if (rc) return rc;
  const int64_t nqh = (k + 1) / 64 + 1;
  lm.bits(b->qz, n3, k + 2, b->qh, nqh, 64 * nqh, 0);
  // r^ = x - q^ m in [-m, 4m): its low k + 3 bits from a low product, sign-extended
  rc = tm_mul_operand(reinterpret_cast<uint64_t*>(b->t), reinterpret_cast<uint64_t*>(b->qz),
                      b->opM, stream, nullptr);
  if (rc) return rc;
  lm.bits(b->xl, n3, k + 3, dx, nx, 2 * k, 0);
  lm.lop(tmul::sum(b->rr, Wr, b->xl, n3, b->t, n3, true));
  lm.sext(b->rr, Wr, k + 3);
  for (int i = 0; i < 2; ++i) {                     // r < 0: r += m, q -= 1
    tmul::LopArgs a = tmul::sum(b->rr, Wr, b->rr, Wr, b->mW, Wr, false);
    a.cond = tmul::kCondANeg;
    a.delta = &lm.flags->delta;
    a.dinc = -1;
    lm.lop(a);
  }
  for (int i = 0; i < 4; ++i) {                     // r >= m: r -= m, q += 1
    tmul::LopArgs a = tmul::sum(b->rr, Wr, b->rr, Wr, b->mW, Wr, true);
    a.cond = tmul::kCondResultNonneg;
    a.delta = &lm.flags->delta;
    a.dinc = 1;
    lm.lop(a);
  }
  for (int neg = 0; neg < 2; ++neg) {               // 0 <= r < m must hold now
    tmul::LopArgs a = tmul::sum(b->rr, Wr, b->rr, Wr, b->mW, Wr, neg == 1);
    a.cond = neg ? tmul::kCondResultNonneg : tmul::kCondANeg;
    a.delta = &lm.flags->fail;
    a.dinc = 1;
    lm.lop(a);
  }
  if (q) {
    tmul::LopArgs f{};
    f.a = b->qz; f.na = n3; f.b_small = &lm.flags->delta; f.out = b->qq; f.W = Wr;
    f.cond = tmul::kCondAlways;
    lm.lop(f);
    lm.bits(reinterpret_cast<u64*>(q), tmul::L(k + 1), k + 1, b->qq, Wr, 64 * Wr, 0);
  }
  if (r) lm.bits(reinterpret_cast<u64*>(r), tmul::L(k), k, b->rr, Wr, 64 * Wr, 0);
  rc = tmul::cuda_rc(cudaGetLastError());
  if (rc || !rep) return rc;
  // the report: the high product's plan; e_max the larger of the two bounds, the
  // margin the largest rounding distance of both products
  *rep = b->plan_hi;
  rep->e_max = std::max(b->plan_hi.e_max, b->plan_lo.e_max);
  rep->workspace_bytes = std::max(b->plan_hi.workspace_bytes, b->plan_lo.workspace_bytes);
  rc = tm_stream_status(stream, rep);
  tmul::Flags fl{};
  int rc2 = tmul::cuda_rc(cudaMemcpyAsync(&fl, lm.flags, sizeof(fl), cudaMemcpyDeviceToHost, s));
  if (!rc2) rc2 = tmul::cuda_rc(cudaStreamSynchronize(s));
  if (rc2) return rc2;
  if (fl.fail) {
    rep->status = TM_EPRECISION;
    return TM_EPRECISION;
  }
  return rc;
}

int tm_barrett_destroy(tm_barrett* b) {
  if (!b) return TM_OK;
  cudaDeviceSynchronize();
  barrett_free(b);
  return TM_OK;
}

}  // extern "C"
