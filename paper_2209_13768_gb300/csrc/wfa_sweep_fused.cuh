// sweep_col2<S>: two explicit steps per pass (Sec. 1.1.1, Eq. expl_form,
// applied twice) with uniform k: temporal blocking on the column-march
// design, so each pass reads and writes the field once for two steps.
//
// A block of 16 x 18 threads owns a 64 x 16 output tile and marches z. Stage
// 1 (the first step) runs on the tile plus a one-cell ring: thread row ty
// holds tile row ty - 1 (rows -1 .. 16), four x cells per thread, and the
// threads of the two ring rows also take the ring column cells (x = -1 and
// x = 64) of the 16 tile rows. Stage 1 writes its plane into a shared ring of
// three planes; after one barrier per plane, stage 2 (the second step) updates
// the tile one plane behind, reading x / y neighbours from shared memory and
// z neighbours from its own register queue. Both stages evaluate the same
// fixed per-cell expression as every other kernel (boundary faces by select,
// held cells, zero-flux self terms), so the field after a pass is bitwise the
// field after two single steps. Cells outside the domain on a non-periodic
// axis keep their input value in stage 1 (they are never read there).
#pragma once

#include "wfa_sweep_col.cuh"

namespace wfa {

constexpr int F2_TX = 16, F2_TY = 18;   // threads; rows -1 .. 16 of the tile
constexpr int F2_W = 72;                 // shared row: x = -4 .. 67, x = 0 at index 4 (16-byte aligned)
constexpr int F2_PLANE = F2_TY * F2_W;
constexpr int F2_BLOCKS = 3;             // blocks per SM the register budget targets

template <typename S>
__global__ void __launch_bounds__(F2_TX * F2_TY, F2_BLOCKS) sweep_col2(const __grid_constant__ SweepArgs a) {
    const SweepCoef& c = a.c;
    __shared__ __align__(16) float s1[3][F2_PLANE];   // stage-1 planes q mod 3

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * 64, y0 = blockIdx.y * 16;
    const int gx = x0 + 4 * tx;              // own cells gx .. gx + 3
    const int gy = y0 - 1 + ty;              // own row (stage 1), -1 .. ny + 15
    const long long sy = c.sy, sz = c.sz;
    const S* __restrict__ tin = (const S*)a.tin;
    S* __restrict__ tout = (S*)a.tout;

    // stage 1 is needed on x in [-1, nx], y in [-1, ny] (the ring of the domain)
    const bool act1 = gx <= c.n[0] && gy <= c.n[1];
    // ring column cell of the two ring rows: x0 - 1 (ty = 0) or x0 + 64 (ty = 17), tile row tx
    const bool ringt = ty == 0 || ty == F2_TY - 1;
    const int rx = ty == 0 ? x0 - 1 : x0 + 64, ry = y0 + tx;
    const bool act_r = ringt && ry <= c.n[1] && rx <= c.n[0];
    const int rcol = ty == 0 ? 3 : 4 + 64;   // its shared column
    // stage 2: tile rows (ty 1 .. 16) inside the domain
    const bool act2 = ty >= 1 && ty <= 16 && gy < c.n[1] && gx < c.n[0];

    // x / y faces of this thread's cells never change along z
    const bool perx = c.periodic[0], pery = c.periodic[1];
    // (self terms and held layers belong to boundary cells only, which
    // inner_xy already excludes on non-periodic axes)
    const bool inner_xy = (perx || (gx > 0 && gx + 3 < c.n[0] - 1)) && (pery || (gy > 0 && gy < c.n[1] - 1)) &&
                          gx + 3 < c.n[0];
    bool out_x[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) out_x[i] = !perx && (gx + i < 0 || gx + i >= c.n[0]);
    const bool out_y = !pery && (gy < 0 || gy >= c.n[1]);

    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, c.n[2]);
    const S* tcol = tin + (long long)gy * sy + gx;   // plane p at tcol + p * sz
    const S* rcolp = tin + (long long)ry * sy + rx;

    // stage-1 input queue (planes q-1, q) and stage-1 output queue (planes q-2, q-1)
    float tm[4], tc[4], sm[4], sc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) tm[i] = tc[i] = sm[i] = sc[i] = 0.0f;
    if (act1) {
        ldg4<S, false>(tcol + (long long)(z0 - 2) * sz, tm);
        ldg4<S, false>(tcol + (long long)(z0 - 1) * sz, tc);
    }
    float rm = 0.0f, rc = 0.0f;   // ring cell input queue
    if (act_r) {
        rm = ldg1<S, false>(rcolp + (long long)(z0 - 2) * sz);
        rc = ldg1<S, false>(rcolp + (long long)(z0 - 1) * sz);
    }

    for (int q = z0 - 1; q <= z1; ++q) {
        float* sp = s1[(q + 3) % 3];
        const bool zin = c.periodic[2] || (q > 0 && q < c.n[2] - 1);
        const bool zout = !c.periodic[2] && (q < 0 || q >= c.n[2]);
        // ring cell inputs first: their latency overlaps the main stage-1 work
        float rz = 0.0f, r_xm = 0.0f, r_xp = 0.0f, r_ym = 0.0f, r_yp = 0.0f;
        if (act_r) {
            const S* rp = rcolp + (long long)q * sz;
            rz = ldg1<S, false>(rp + sz);
            r_xm = ldg1<S, false>(rp - 1);
            r_xp = ldg1<S, false>(rp + 1);
            r_ym = ldg1<S, false>(rp - sy);
            r_yp = ldg1<S, false>(rp + sy);
        }
        // ---- stage 1 at plane q
        float sn[4];
        if (act1) {
            const S* tp = tcol + (long long)q * sz;
            float tz[4], ym[4], yp[4];
            ldg4<S, false>(tp + sz, tz);
            if ((tx & 7) == 0) prefetch_l2(tp + 3 * sz);
            ldg4<S, false>(tp - sy, ym);
            ldg4<S, false>(tp + sy, yp);
            const float xm = ldg1<S, false>(tp - 1), xp = ldg1<S, false>(tp + 4);
            if (inner_xy && zin) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    sn[i] = storage_round<S>(uniform_inner(c, tc[i], i == 0 ? xm : tc[i - 1], i == 3 ? xp : tc[i + 1],
                                                           ym[i], yp[i], tm[i], tz[i]));
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float v = uniform_cell(c, tc[i], i == 0 ? xm : tc[i - 1], i == 3 ? xp : tc[i + 1], ym[i],
                                                 yp[i], tm[i], tz[i], gx + i, gy, q);
                    sn[i] = (out_x[i] || out_y || zout) ? tc[i] : storage_round<S>(v);
                }
            }
            Vec4<float>::store(sp + ty * F2_W + 4 + 4 * tx, sn);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                tm[i] = tc[i];
                tc[i] = tz[i];
            }
        }
        if (act_r) {
            const float v = uniform_cell(c, rc, r_xm, r_xp, r_ym, r_yp, rm, rz, rx, ry, q);
            sp[(tx + 1) * F2_W + rcol] = outside_np(c, rx, ry, q) ? rc : storage_round<S>(v);
            rm = rc;
            rc = rz;
        }
        __syncthreads();
        // ---- stage 2 at plane q - 1 (stage-1 planes q-2, q-1, q)
        const int p = q - 1;
        if (act2 && p >= z0) {
            const float* pp = s1[(p + 3) % 3];
            const int o = ty * F2_W + 4 + 4 * tx;
            float ym[4], yp[4];
            Vec4<float>::load(pp + o - F2_W, ym);
            Vec4<float>::load(pp + o + F2_W, yp);
            const float xm = pp[o - 1], xp = pp[o + 4];
            float out[4];
            const bool pin = c.periodic[2] || (p > 0 && p < c.n[2] - 1);
            if (inner_xy && pin) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    out[i] = uniform_inner(c, sc[i], i == 0 ? xm : sc[i - 1], i == 3 ? xp : sc[i + 1], ym[i], yp[i],
                                           sm[i], sn[i]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    out[i] = uniform_cell(c, sc[i], i == 0 ? xm : sc[i - 1], i == 3 ? xp : sc[i + 1], ym[i], yp[i],
                                          sm[i], sn[i], gx + i, gy, p);
            }
            S* op = tout + (long long)p * sz + (long long)gy * sy + gx;
            if (gx + 3 < c.n[0]) {
                float r4[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) r4[i] = out[i];
                Vec4<S>::store(op, r4);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (gx + i < c.n[0]) op[i] = from_f32<S>(out[i]);
            }
        }
        if (act1) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                sm[i] = sc[i];
                sc[i] = sn[i];
            }
        }
    }
}

// One pass of two steps; then the periodic twins of the written buffer.
template <typename S>
cudaError_t col2_launch(const SweepArgs& a_in, cudaStream_t st, int nsm, const cudaEvent_t* ev) {
    SweepArgs a = a_in;
    const dim3 block(F2_TX, F2_TY);
    const int gxb = (a.c.n[0] + 63) / 64, gyb = (a.c.n[1] + 15) / 16;
    const long long cols = (long long)gxb * gyb, resident = (long long)nsm * F2_BLOCKS;
    // z chunks of at least 32 planes (each chunk recomputes two stage-1
    // planes), shorter only when that would leave SMs idle
    int nch = (int)std::max<long long>(1, resident * 8 / cols);
    int cap = std::max(1, a.c.n[2] / 32);
    if (cols * cap < resident) cap = std::max(1, a.c.n[2] / 4);
    nch = std::min(nch, cap);
    a.zchunk = (a.c.n[2] + nch - 1) / nch;
    nch = (a.c.n[2] + a.zchunk - 1) / a.zchunk;
    if (ev) cudaEventRecord(ev[0], st);
    sweep_col2<S><<<dim3(gxb, gyb, nch), block, 0, st>>>(a);
    if (ev) cudaEventRecord(ev[1], st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int ax = 0; ax < 3; ++ax) {
        if (!a.c.periodic[ax]) continue;
        const int b = ax == 0 ? 1 : 0, d = ax == 2 ? 1 : 2;
        const long long total = 2LL * HALO * (a.c.n[b] + 2 * HALO) * (a.c.n[d] + 2 * HALO);
        const int nb = (int)std::min<long long>((total + 255) / 256, (long long)nsm * 8);
        twin_copy<S><<<nb, 256, 0, st>>>(a.c, (S*)a.tout, ax);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace wfa
