// Standalone probe of the assignment kernel's dense-row phase, measured in
// isolation (a program of its own, not part of the library). Persistent CTAs score one
// object at a time: the object's nd rows of a BF16 row matrix are read with
// 16-byte loads (eight rows in flight per thread), accumulated in FP32 per
// position and added into a shared fixed-point score vector, followed by a
// top-1 pass that also zeroes it, as in the library's loop. Variants: mixed
// BF16 x BF16 -> FP32 FMAs (object value rounded to BF16), L1::no_allocate
// loads, 32-byte loads, the top-1 taken from registers without atomics, and
// 256 / 1024-thread CTAs. Synthetic input: 300,000 objects x 40 distinct rows
// of a 2,400 x 20,000 matrix (rows drawn with weight 1/(r+1)^0.8), seeded.
//
// Build and run on one GB300:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 -o dense_rows dense_rows.cu && ./dense_rows
// Every index stays inside its buffer: KPAD and ND are multiples of 8, rows
// start at multiples of 32 bytes, and positions p + 8 (p + 16 for 32-byte
// loads) never pass KPAD.
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>
#include <algorithm>
#include <cmath>
#include <cstring>

constexpr int KPAD = 20000;  // multiple of 8
constexpr int R = 2400;
constexpr int ND = 40;
constexpr int NOBJ = 300000;

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e_), __LINE__); exit(1); } } while (0)

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

__device__ __forceinline__ uint4 ld16(const uint16_t *p) {
    uint4 r;
    asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}
__device__ __forceinline__ uint4 ld16_na(const uint16_t *p) {
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}
struct U8 { uint32_t w[8]; };
__device__ __forceinline__ U8 ld32(const uint16_t *p) {
    U8 r;
    asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3]), "=r"(r.w[4]), "=r"(r.w[5]), "=r"(r.w[6]),
                   "=r"(r.w[7]) : "l"(p));
    return r;
}
__device__ __forceinline__ void fma8(const uint4 &r, float v, float *acc) {
    acc[0] = fmaf(bf_lo(r.x), v, acc[0]);
    acc[1] = fmaf(bf_hi(r.x), v, acc[1]);
    acc[2] = fmaf(bf_lo(r.y), v, acc[2]);
    acc[3] = fmaf(bf_hi(r.y), v, acc[3]);
    acc[4] = fmaf(bf_lo(r.z), v, acc[4]);
    acc[5] = fmaf(bf_hi(r.z), v, acc[5]);
    acc[6] = fmaf(bf_lo(r.w), v, acc[6]);
    acc[7] = fmaf(bf_hi(r.w), v, acc[7]);
}
__device__ __forceinline__ void mfma2(uint32_t w, uint16_t vb, float &a0, float &a1) {
    asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\t"
        "fma.rn.f32.bf16 %0, l, %3, %0;\n\tfma.rn.f32.bf16 %1, h, %3, %1;\n\t}"
        : "+f"(a0), "+f"(a1) : "r"(w), "h"(vb));
}

// VAR 0: as the library (U = 8 loads of 16 B, unpack + FMA, atomics, top-1 pass)
// VAR 1: mixed-precision FMA (object value rounded to BF16)
// VAR 2: no L1 allocation on the row loads
// VAR 3: 32-byte loads, 16 positions per thread, U = 4
// VAR 4: fused: no atomics, the top-1 is taken from the registers (rho read for the sparse part)
template <int T, int VAR>
__global__ void __launch_bounds__(T, 1024 / T) kern(const uint16_t *__restrict__ dense, const int *__restrict__ orow,
                                                     const float *__restrict__ ov, unsigned long long *work,
                                                     int *label) {
    extern __shared__ __align__(16) uint32_t rho[];
    __shared__ int2 s_dense[ND];
    __shared__ long long s_obj;
    __shared__ unsigned long long wbest[T / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int p = tid; p < KPAD; p += T) rho[p] = 0u;
    __syncthreads();
    for (;;) {
        if (tid == 0) s_obj = (long long)atomicAdd(work, 1ull);
        __syncthreads();
        const long long o = s_obj;
        if (o >= NOBJ) break;
        if (tid < ND) s_dense[tid] = make_int2(orow[o * ND + tid], __float_as_int(ov[o * ND + tid] * 2147483648.0f));
        __syncthreads();
        unsigned long long best = 0ull;
        if constexpr (VAR == 3) {
            constexpr int U = 4;
            for (int base = 0; base < KPAD; base += 16 * T) {
                const int p = base + 16 * tid;
                if (p >= KPAD) continue;
                const bool two = p + 8 < KPAD;  // KPAD is a multiple of 8, not of 16
                float acc[16];
#pragma unroll
                for (int m = 0; m < 16; ++m) acc[m] = 0.f;
                for (int d = 0; d < ND; d += U) {
                    U8 r[U];
#pragma unroll
                    for (int q = 0; q < U; ++q) {
                        const uint16_t *ptr = dense + (size_t)s_dense[d + q].x * KPAD + p;
                        if (two) r[q] = ld32(ptr);
                        else {
                            const uint4 h = ld16(ptr);
                            r[q].w[0] = h.x; r[q].w[1] = h.y; r[q].w[2] = h.z; r[q].w[3] = h.w;
                            r[q].w[4] = r[q].w[5] = r[q].w[6] = r[q].w[7] = 0u;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < U; ++q) {
                        const float v = __int_as_float(s_dense[d + q].y);
                        fma8(make_uint4(r[q].w[0], r[q].w[1], r[q].w[2], r[q].w[3]), v, acc);
                        fma8(make_uint4(r[q].w[4], r[q].w[5], r[q].w[6], r[q].w[7]), v, acc + 8);
                    }
                }
#pragma unroll
                for (int m = 0; m < 16; ++m)
                    if ((m < 8 || two) && acc[m] > 0.f) atomicAdd(rho + p + m, __float2uint_ru(acc[m]));
            }
        } else {
            constexpr int U = 8;
            for (int base = 0; base < KPAD; base += 8 * T) {
                const int p = base + 8 * tid;
                if (p >= KPAD) continue;
                float acc[8];
#pragma unroll
                for (int m = 0; m < 8; ++m) acc[m] = 0.f;
                for (int d = 0; d < ND; d += U) {
                    uint4 r[U];
#pragma unroll
                    for (int q = 0; q < U; ++q) {
                        const uint16_t *ptr = dense + (size_t)s_dense[d + q].x * KPAD + p;
                        r[q] = VAR == 2 ? ld16_na(ptr) : ld16(ptr);
                    }
#pragma unroll
                    for (int q = 0; q < U; ++q) {
                        const float v = __int_as_float(s_dense[d + q].y);
                        if constexpr (VAR == 1) {
                            const uint16_t vb = (uint16_t)(__float_as_uint(v) >> 16);
                            mfma2(r[q].x, vb, acc[0], acc[1]);
                            mfma2(r[q].y, vb, acc[2], acc[3]);
                            mfma2(r[q].z, vb, acc[4], acc[5]);
                            mfma2(r[q].w, vb, acc[6], acc[7]);
                        } else {
                            fma8(r[q], v, acc);
                        }
                    }
                }
                if constexpr (VAR == 4) {
#pragma unroll
                    for (int m = 0; m < 8; ++m) {
                        const uint32_t s = rho[p + m] + (acc[m] > 0.f ? __float2uint_ru(acc[m]) : 0u);
                        const unsigned long long key = ((unsigned long long)s << 32) | (uint32_t)(~(p + m));
                        best = key > best ? key : best;
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < 8; ++m)
                        if (acc[m] > 0.f) atomicAdd(rho + p + m, __float2uint_ru(acc[m]));
                }
            }
        }
        if constexpr (VAR != 4) {
            __syncthreads();
            for (int p = tid; p < KPAD; p += T) {
                const unsigned long long key = ((unsigned long long)rho[p] << 32) | (uint32_t)(~p);
                best = key > best ? key : best;
                rho[p] = 0u;
            }
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, best, s);
            best = y > best ? y : best;
        }
        if (lane == 0) wbest[warp] = best;
        __syncthreads();
        if (tid == 0) {
            unsigned long long b = wbest[0];
            for (int w = 1; w < T / 32; ++w) b = wbest[w] > b ? wbest[w] : b;
            label[o] = (int)(~(uint32_t)b);
        }
    }
}

template <int T, int VAR>
float run(const char *name, const uint16_t *d_dense, const int *d_row, const float *d_v, unsigned long long *d_work,
          int *d_label, int nsm, std::vector<int> &lab) {
    auto k = kern<T, VAR>;
    const int smem = KPAD * 4;
    CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, T, smem));
    float best = 1e30f;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int rep = 0; rep < 4; ++rep) {
        CK(cudaMemset(d_work, 0, 8));
        CK(cudaEventRecord(e0));
        k<<<nsm * per_sm, T, smem>>>(d_dense, d_row, d_v, d_work, d_label);
        CK(cudaEventRecord(e1));
        CK(cudaEventSynchronize(e1));
        CK(cudaGetLastError());
        float ms;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) best = std::min(best, ms);
    }
    lab.resize(NOBJ);
    CK(cudaMemcpy(lab.data(), d_label, sizeof(int) * NOBJ, cudaMemcpyDeviceToHost));
    const double ent = (double)NOBJ * ND * KPAD;
    printf("%-34s T=%4d ctas/SM=%d  %8.2f ms  %.3g entries/s  %.2f TB/s\n", name, T, per_sm, best, ent / best * 1e3,
           ent * 2 / best * 1e3 / 1e12);
    return best;
}

int main() {
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, 0));
    const int nsm = prop.multiProcessorCount;
    std::mt19937_64 rng(7);
    std::vector<uint16_t> h_dense((size_t)R * KPAD);
    std::uniform_real_distribution<float> uf(0.f, 0.05f);
    for (auto &x : h_dense) {
        const float f = (rng() % 4 == 0) ? 0.f : uf(rng);
        uint32_t b;
        memcpy(&b, &f, 4);
        x = (uint16_t)(b >> 16);
    }
    std::vector<double> w(R);
    for (int r = 0; r < R; ++r) w[r] = 1.0 / pow(r + 1.0, 0.8);
    std::discrete_distribution<int> pick(w.begin(), w.end());
    std::vector<int> h_row((size_t)NOBJ * ND);
    std::vector<float> h_v((size_t)NOBJ * ND);
    std::uniform_real_distribution<float> vf(0.01f, 0.2f);
    for (int o = 0; o < NOBJ; ++o) {
        int n = 0;
        while (n < ND) {
            const int r = pick(rng);
            bool dup = false;
            for (int q = 0; q < n; ++q) dup |= h_row[(size_t)o * ND + q] == r;
            if (!dup) {
                h_row[(size_t)o * ND + n] = r;
                h_v[(size_t)o * ND + n] = vf(rng);
                ++n;
            }
        }
    }
    uint16_t *d_dense;
    int *d_row, *d_label;
    float *d_v;
    unsigned long long *d_work;
    CK(cudaMalloc(&d_dense, h_dense.size() * 2));
    CK(cudaMalloc(&d_row, h_row.size() * 4));
    CK(cudaMalloc(&d_v, h_v.size() * 4));
    CK(cudaMalloc(&d_label, NOBJ * 4));
    CK(cudaMalloc(&d_work, 8));
    CK(cudaMemcpy(d_dense, h_dense.data(), h_dense.size() * 2, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_row, h_row.data(), h_row.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_v, h_v.data(), h_v.size() * 4, cudaMemcpyHostToDevice));
    std::vector<int> l0, l;
    run<512, 0>("V0 library form", d_dense, d_row, d_v, d_work, d_label, nsm, l0);
    auto same = [&](const char *n) {
        size_t d = 0;
        for (int i = 0; i < NOBJ; ++i) d += l[i] != l0[i];
        printf("    %s: %zu labels differ from V0\n", n, d);
    };
    run<512, 1>("V1 mixed bf16 FMA", d_dense, d_row, d_v, d_work, d_label, nsm, l); same("V1");
    run<512, 2>("V2 L1::no_allocate", d_dense, d_row, d_v, d_work, d_label, nsm, l); same("V2");
    run<512, 3>("V3 32-byte loads, U=4", d_dense, d_row, d_v, d_work, d_label, nsm, l); same("V3");
    run<512, 4>("V4 fused top-1, no atomics", d_dense, d_row, d_v, d_work, d_label, nsm, l); same("V4");
    run<1024, 0>("V0 library form", d_dense, d_row, d_v, d_work, d_label, nsm, l); same("V0/1024");
    run<256, 0>("V0 library form", d_dense, d_row, d_v, d_work, d_label, nsm, l); same("V0/256");
    return 0;
}
