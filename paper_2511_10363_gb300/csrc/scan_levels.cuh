// scan_levels.cuh -- the all-prefix-sum algorithms of Sec. II of
// arXiv 2511.10363 run level by level over element buffers in device memory:
// Hillis-Steele (Alg. 1), Blelloch (Alg. 2), the in-place Ladner-Fischer
// circuit (Alg. 3) and the hybrid of Sengupta et al. (Alg. sengupta).  One launch per level; each launch covers the level's
// independent operator applications with a grid-stride loop.
//
// Elements are stored structure-of-arrays by scalar component,
// buf[c * Tpad + i], so that each component load of a warp is one
// coalesced 128-byte line.  T is padded to the next power of two Tpad with
// neutral elements placed after the last scan position (Sec. II).
// Paper index i (1-based) is buffer index i - 1.
#pragma once

#include "scan_dlb.cuh"

namespace kfs {

template <class X, typename R>
KF_D void load_soa(X &x, const R *buf, int64_t stride, int64_t i) {
#pragma unroll
    for (int c = 0; c < X::SIZE; ++c) x.v[c] = buf[c * stride + i];
}
template <class X, typename R>
KF_D void store_soa(const X &x, R *buf, int64_t stride, int64_t i) {
#pragma unroll
    for (int c = 0; c < X::SIZE; ++c) buf[c * stride + i] = x.v[c];
}

KF_D int64_t gtid() { return int64_t(blockIdx.x) * blockDim.x + threadIdx.x; }
KF_D int64_t gstride() { return int64_t(gridDim.x) * blockDim.x; }

// a[i] = element at scan position i (neutral element past the end); b, when
// given, receives a copy (Blelloch's "b <- copy(a)").
template <class P>
__global__ void lv_build(const __grid_constant__ typename P::Args args, typename P::R *a, typename P::R *b,
                         int64_t Tpad) {
    using Elem = typename P::Elem;
    const int64_t total = P::total(args);
    for (int64_t i = gtid(); i < Tpad; i += gstride()) {
        Elem e;
        if (i < total) {
            SegCursor cur = P::cursor(args, i);
            P::build(args, i, cur, in_rec_direct<P>(args, global_index<P>(args, i)), e);
        } else {
            set_identity(e);
        }
        store_soa(e, a, Tpad, i);
        if (b) store_soa(e, b, Tpad, i);
    }
}

// Alg. 1, one level: dst_j = src_{j-2^d} (x) src_j for j > 2^d, dst_j = src_j otherwise.
template <class P>
__global__ void lv_hillis_steele(const typename P::R *src, typename P::R *dst, int64_t Tpad, int64_t off) {
    using Elem = typename P::Elem;
    for (int64_t j = gtid(); j < Tpad; j += gstride()) {
        Elem y;
        load_soa(y, src, Tpad, j);
        if (j >= off) {
            Elem x, o;
            load_soa(x, src, Tpad, j - off);
            P::combine(x, y, o);
            store_soa(o, dst, Tpad, j);
        } else {
            store_soa(y, dst, Tpad, j);
        }
    }
}

// Alg. sengupta, reduce pass: dst_i = src_{2i-1} (x) src_{2i} (1-based),
// src of length ls, dst of length ld = ls / 2 (each its own stride).
template <class P>
__global__ void lv_sg_reduce(const typename P::R *src, int64_t ls, typename P::R *dst, int64_t ld) {
    using Elem = typename P::Elem;
    for (int64_t i = gtid(); i < ld; i += gstride()) {
        Elem x, y, o;
        load_soa(x, src, ls, 2 * i);
        load_soa(y, src, ls, 2 * i + 1);
        P::combine(x, y, o);
        store_soa(o, dst, ld, i);
    }
}

// Alg. sengupta, down-sweep of one level: with `up` the scanned level above,
// cur_i = up_{i/2} for even i and up_{(i-1)/2} (x) cur_i for odd i > 1
// (1-based; cur_1 stays).
template <class P>
__global__ void lv_sg_down(const typename P::R *up, int64_t lu, typename P::R *cur, int64_t lc) {
    using Elem = typename P::Elem;
    for (int64_t i = gtid() + 1; i < lc; i += gstride()) {   // 0-based; index 0 stays
        Elem x;
        if (i & 1) {          // 1-based i + 1 even
            load_soa(x, up, lu, (i - 1) / 2);
            store_soa(x, cur, lc, i);
        } else {              // 1-based i + 1 odd, > 1
            Elem y, o;
            load_soa(x, up, lu, i / 2 - 1);
            load_soa(y, cur, lc, i);
            P::combine(x, y, o);
            store_soa(o, cur, lc, i);
        }
    }
}

// Up-sweep level d (Algs. 2 and 3): a_k <- a_j (x) a_k, j = i + 2^d, k = i + 2^{d+1},
// i = 0, 2^{d+1}, ... (1-based paper indices).
template <class P>
__global__ void lv_upsweep(typename P::R *a, int64_t Tpad, int d) {
    using Elem = typename P::Elem;
    const int64_t h = int64_t(1) << d, w = h << 1, npairs = Tpad / w;
    for (int64_t t = gtid(); t < npairs; t += gstride()) {
        const int64_t j = t * w + h - 1, k = t * w + w - 1;
        Elem x, y, o;
        load_soa(x, a, Tpad, j);
        load_soa(y, a, Tpad, k);
        P::combine(x, y, o);
        store_soa(o, a, Tpad, k);
    }
}

// Alg. 2: a_T <- neutral element.
template <class P>
__global__ void lv_set_identity(typename P::R *a, int64_t Tpad, int64_t i) {
    using Elem = typename P::Elem;
    if (gtid() == 0) {
        Elem e;
        set_identity(e);
        store_soa(e, a, Tpad, i);
    }
}

// Alg. 2 down-sweep level d: t <- a_j; a_j <- a_k; a_k <- a_k (x) t.
template <class P>
__global__ void lv_blelloch_down(typename P::R *a, int64_t Tpad, int d) {
    using Elem = typename P::Elem;
    const int64_t h = int64_t(1) << d, w = h << 1, npairs = Tpad / w;
    for (int64_t t = gtid(); t < npairs; t += gstride()) {
        const int64_t j = t * w + h - 1, k = t * w + w - 1;
        Elem x, y, o;
        load_soa(x, a, Tpad, j);
        load_soa(y, a, Tpad, k);
        P::combine(y, x, o);
        store_soa(y, a, Tpad, j);
        store_soa(o, a, Tpad, k);
    }
}

// Alg. 2 final pass: a_i <- a_i (x) b_i.
template <class P>
__global__ void lv_blelloch_final(typename P::R *a, const typename P::R *b, int64_t Tpad) {
    using Elem = typename P::Elem;
    for (int64_t i = gtid(); i < Tpad; i += gstride()) {
        Elem x, y, o;
        load_soa(x, a, Tpad, i);
        load_soa(y, b, Tpad, i);
        P::combine(x, y, o);
        store_soa(o, a, Tpad, i);
    }
}

// Alg. 3 down-sweep level d: a_j <- a_i (x) a_j, j = i + 2^d, i = 2^{d+1}, 2*2^{d+1}, ...
template <class P>
__global__ void lv_lafi_down(typename P::R *a, int64_t Tpad, int d) {
    using Elem = typename P::Elem;
    const int64_t h = int64_t(1) << d, w = h << 1, n = Tpad / w - 1;
    for (int64_t t = gtid(); t < n; t += gstride()) {
        const int64_t i = (t + 1) * w - 1, j = i + h;
        Elem x, y, o;
        load_soa(x, a, Tpad, i);
        load_soa(y, a, Tpad, j);
        P::combine(x, y, o);
        store_soa(o, a, Tpad, j);
    }
}

// Extraction (Algs. pkf / prts / ptf "Extract the results"): the carry of
// prefix s_p is emitted.  With a log-likelihood, s_p is instead reached from
// s_{p-1} by one application of a_p, which yields the innovation term.
template <class P, int THREADS>
__global__ void __launch_bounds__(THREADS) lv_extract(const __grid_constant__ typename P::Args args,
                                                      const typename P::R *a, int64_t Tpad, double *ll_part,
                                                      int *counter, double *ll_out) {
    using Elem = typename P::Elem;
    using Carry = typename P::Carry;
    constexpr int NW = THREADS / 32;
    __shared__ double s_ll[NW];
    __shared__ int s_last;
    const int64_t total = P::total(args);
    double ll = 0.0;
    for (int64_t p = gtid(); p < total; p += gstride()) {
        SegCursor cur = P::cursor(args, p);
        const int64_t g = global_index<P>(args, p);
        const typename P::R *in = in_rec_direct<P>(args, g);
        typename P::R *o1 = out_rec_direct<P>(args, 0, g), *o2 = out_rec_direct<P>(args, 1, g),
                      *o3 = out_rec_direct<P>(args, 2, g);
        if (ll_out) {
            Carry c;
            set_zero(c);
            if (p > 0) {
                Elem s;
                load_soa(s, a, Tpad, p - 1);
                P::carry_of(s, c);
            }
            Elem e;
            P::build(args, p, cur, in, e);
            ll += P::step(args, p, cur, c, e, in, o1, o2, o3);
        } else {
            Elem s;
            Carry c;
            load_soa(s, a, Tpad, p);
            P::carry_of(s, c);
            P::emit(args, p, cur, c, in, o1, o2, o3);
        }
    }
    if (!ll_out) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) ll += __shfl_down_sync(0xffffffffu, ll, s);
    if (lane == 0) s_ll[warp] = ll;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < NW; ++w) t += s_ll[w];
        ll_part[blockIdx.x] = t;
        __threadfence();
        s_last = (atomicAdd(counter, 1) == int(gridDim.x) - 1);
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        double t = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(ll_part + b);
        *ll_out = t;
    }
}

}  // namespace kfs
