// Multi-word additions on the hardware carry chain: one add per 32-bit word
// (word 0 lowest).  add(s, a, b): s = a + b, returns the carry out of the
// top word.  inc(s, c): s += c for c in {0, 1} (the carry out is dropped).
#pragma once

#include <stdint.h>

namespace msa {

template <int N>
struct CarryChain;

template <>
struct CarryChain<1> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[1], const uint32_t (&a)[1],
                                                   const uint32_t (&b)[1]) {
        uint32_t c;
        asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, 0, 0;"
            : "=r"(s[0]), "=r"(c)
            : "r"(a[0]), "r"(b[0]));
        return c;
    }
    static __device__ __forceinline__ void inc(uint32_t (&s)[1], uint32_t ci) {
        asm("add.u32 %0, %0, %1;"
            : "+r"(s[0])
            : "r"(ci));
    }
};

template <>
struct CarryChain<2> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[2], const uint32_t (&a)[2],
                                                   const uint32_t (&b)[2]) {
        uint32_t c;
        asm("add.cc.u32 %0, %3, %5;\n\taddc.cc.u32 %1, %4, %6;\n\taddc.u32 %2, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(c)
            : "r"(a[0]), "r"(a[1]), "r"(b[0]), "r"(b[1]));
        return c;
    }
    static __device__ __forceinline__ void inc(uint32_t (&s)[2], uint32_t ci) {
        asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, 0;"
            : "+r"(s[0]), "+r"(s[1])
            : "r"(ci));
    }
};

template <>
struct CarryChain<3> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[3], const uint32_t (&a)[3],
                                                   const uint32_t (&b)[3]) {
        uint32_t c;
        asm("add.cc.u32 %0, %4, %7;\n\taddc.cc.u32 %1, %5, %8;\n\taddc.cc.u32 %2, %6, %9;\n\taddc.u32 %3, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(c)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(b[0]), "r"(b[1]), "r"(b[2]));
        return c;
    }
    static __device__ __forceinline__ void inc(uint32_t (&s)[3], uint32_t ci) {
        asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.u32 %2, %2, 0;"
            : "+r"(s[0]), "+r"(s[1]), "+r"(s[2])
            : "r"(ci));
    }
};

template <>
struct CarryChain<4> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[4], const uint32_t (&a)[4],
                                                   const uint32_t (&b)[4]) {
        uint32_t c;
        asm("add.cc.u32 %0, %5, %9;\n\taddc.cc.u32 %1, %6, %10;\n\taddc.cc.u32 %2, %7, %11;\n\taddc.cc.u32 %3, %8, %12;\n\taddc.u32 %4, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(c)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]));
        return c;
    }
    static __device__ __forceinline__ void inc(uint32_t (&s)[4], uint32_t ci) {
        asm("add.cc.u32 %0, %0, %4;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.cc.u32 %2, %2, 0;\n\taddc.u32 %3, %3, 0;"
            : "+r"(s[0]), "+r"(s[1]), "+r"(s[2]), "+r"(s[3])
            : "r"(ci));
    }
};

template <>
struct CarryChain<5> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[5], const uint32_t (&a)[5],
                                                   const uint32_t (&b)[5]) {
        uint32_t c;
        asm("add.cc.u32 %0, %6, %11;\n\taddc.cc.u32 %1, %7, %12;\n\taddc.cc.u32 %2, %8, %13;\n\taddc.cc.u32 %3, %9, %14;\n\taddc.cc.u32 %4, %10, %15;\n\taddc.u32 %5, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(c)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]));
        return c;
    }
    static __device__ __forceinline__ void inc(uint32_t (&s)[5], uint32_t ci) {
        asm("add.cc.u32 %0, %0, %5;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.cc.u32 %2, %2, 0;\n\taddc.cc.u32 %3, %3, 0;\n\taddc.u32 %4, %4, 0;"
            : "+r"(s[0]), "+r"(s[1]), "+r"(s[2]), "+r"(s[3]), "+r"(s[4])
            : "r"(ci));
    }
};

template <>
struct CarryChain<6> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[6], const uint32_t (&a)[6],
                                                   const uint32_t (&b)[6]) {
        uint32_t c;
        asm("add.cc.u32 %0, %7, %13;\n\taddc.cc.u32 %1, %8, %14;\n\taddc.cc.u32 %2, %9, %15;\n\taddc.cc.u32 %3, %10, %16;\n\taddc.cc.u32 %4, %11, %17;\n\taddc.cc.u32 %5, %12, %18;\n\taddc.u32 %6, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(c)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]));
        return c;
    }
    static __device__ __forceinline__ void inc(uint32_t (&s)[6], uint32_t ci) {
        asm("add.cc.u32 %0, %0, %6;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.cc.u32 %2, %2, 0;\n\taddc.cc.u32 %3, %3, 0;\n\taddc.cc.u32 %4, %4, 0;\n\taddc.u32 %5, %5, 0;"
            : "+r"(s[0]), "+r"(s[1]), "+r"(s[2]), "+r"(s[3]), "+r"(s[4]), "+r"(s[5])
            : "r"(ci));
    }
};

template <>
struct CarryChain<8> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[8], const uint32_t (&a)[8],
                                                   const uint32_t (&b)[8]) {
        uint32_t c;
        asm("add.cc.u32 %0, %9, %17;\n\taddc.cc.u32 %1, %10, %18;\n\taddc.cc.u32 %2, %11, %19;\n\taddc.cc.u32 %3, %12, %20;\n\taddc.cc.u32 %4, %13, %21;\n\taddc.cc.u32 %5, %14, %22;\n\taddc.cc.u32 %6, %15, %23;\n\taddc.cc.u32 %7, %16, %24;\n\taddc.u32 %8, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(s[7]), "=r"(c)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
        return c;
    }
    static __device__ __forceinline__ void inc(uint32_t (&s)[8], uint32_t ci) {
        asm("add.cc.u32 %0, %0, %8;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.cc.u32 %2, %2, 0;\n\taddc.cc.u32 %3, %3, 0;\n\taddc.cc.u32 %4, %4, 0;\n\taddc.cc.u32 %5, %5, 0;\n\taddc.cc.u32 %6, %6, 0;\n\taddc.u32 %7, %7, 0;"
            : "+r"(s[0]), "+r"(s[1]), "+r"(s[2]), "+r"(s[3]), "+r"(s[4]), "+r"(s[5]), "+r"(s[6]), "+r"(s[7])
            : "r"(ci));
    }
};

template <>
struct CarryChain<10> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[10], const uint32_t (&a)[10],
                                                   const uint32_t (&b)[10]) {
        uint32_t c;
        asm("add.cc.u32 %0, %11, %21;\n\taddc.cc.u32 %1, %12, %22;\n\taddc.cc.u32 %2, %13, %23;\n\taddc.cc.u32 %3, %14, %24;\n\taddc.cc.u32 %4, %15, %25;\n\taddc.cc.u32 %5, %16, %26;\n\taddc.cc.u32 %6, %17, %27;\n\taddc.cc.u32 %7, %18, %28;\n\taddc.cc.u32 %8, %19, %29;\n\taddc.cc.u32 %9, %20, %30;\n\taddc.u32 %10, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(s[7]), "=r"(s[8]), "=r"(s[9]), "=r"(c)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[8]), "r"(a[9]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(b[8]), "r"(b[9]));
        return c;
    }
    static __device__ __forceinline__ void inc(uint32_t (&s)[10], uint32_t ci) {
        asm("add.cc.u32 %0, %0, %10;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.cc.u32 %2, %2, 0;\n\taddc.cc.u32 %3, %3, 0;\n\taddc.cc.u32 %4, %4, 0;\n\taddc.cc.u32 %5, %5, 0;\n\taddc.cc.u32 %6, %6, 0;\n\taddc.cc.u32 %7, %7, 0;\n\taddc.cc.u32 %8, %8, 0;\n\taddc.u32 %9, %9, 0;"
            : "+r"(s[0]), "+r"(s[1]), "+r"(s[2]), "+r"(s[3]), "+r"(s[4]), "+r"(s[5]), "+r"(s[6]), "+r"(s[7]), "+r"(s[8]), "+r"(s[9])
            : "r"(ci));
    }
};

// add_in(s, a, b, cin): s = a + b + cin over N words on the carry chain,
// cin in {0, 1} entered by one add that sets the carry flag (cin + 0xffffffff
// carries exactly when cin = 1); returns the carry out of the top word.
template <int N>
struct CarryChainIn;

template <>
struct CarryChainIn<1> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[1], const uint32_t (&a)[1],
                                                   const uint32_t (&b)[1], uint32_t cin) {
        uint32_t c;
        asm("add.cc.u32 %2, %2, -1;\n\taddc.cc.u32 %0, %3, %4;\n\taddc.u32 %1, 0, 0;"
            : "=r"(s[0]), "=r"(c), "+r"(cin)
            : "r"(a[0]), "r"(b[0]));
        return c;
    }
};

template <>
struct CarryChainIn<2> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[2], const uint32_t (&a)[2],
                                                   const uint32_t (&b)[2], uint32_t cin) {
        uint32_t c;
        asm("add.cc.u32 %3, %3, -1;\n\taddc.cc.u32 %0, %4, %6;\n\taddc.cc.u32 %1, %5, %7;\n\taddc.u32 %2, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(c), "+r"(cin)
            : "r"(a[0]), "r"(a[1]), "r"(b[0]), "r"(b[1]));
        return c;
    }
};

template <>
struct CarryChainIn<3> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[3], const uint32_t (&a)[3],
                                                   const uint32_t (&b)[3], uint32_t cin) {
        uint32_t c;
        asm("add.cc.u32 %4, %4, -1;\n\taddc.cc.u32 %0, %5, %8;\n\taddc.cc.u32 %1, %6, %9;\n\taddc.cc.u32 %2, %7, %10;\n\taddc.u32 %3, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(c), "+r"(cin)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(b[0]), "r"(b[1]), "r"(b[2]));
        return c;
    }
};

template <>
struct CarryChainIn<4> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[4], const uint32_t (&a)[4],
                                                   const uint32_t (&b)[4], uint32_t cin) {
        uint32_t c;
        asm("add.cc.u32 %5, %5, -1;\n\taddc.cc.u32 %0, %6, %10;\n\taddc.cc.u32 %1, %7, %11;\n\taddc.cc.u32 %2, %8, %12;\n\taddc.cc.u32 %3, %9, %13;\n\taddc.u32 %4, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(c), "+r"(cin)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]));
        return c;
    }
};

template <>
struct CarryChainIn<5> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[5], const uint32_t (&a)[5],
                                                   const uint32_t (&b)[5], uint32_t cin) {
        uint32_t c;
        asm("add.cc.u32 %6, %6, -1;\n\taddc.cc.u32 %0, %7, %12;\n\taddc.cc.u32 %1, %8, %13;\n\taddc.cc.u32 %2, %9, %14;\n\taddc.cc.u32 %3, %10, %15;\n\taddc.cc.u32 %4, %11, %16;\n\taddc.u32 %5, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(c), "+r"(cin)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]));
        return c;
    }
};

template <>
struct CarryChainIn<6> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[6], const uint32_t (&a)[6],
                                                   const uint32_t (&b)[6], uint32_t cin) {
        uint32_t c;
        asm("add.cc.u32 %7, %7, -1;\n\taddc.cc.u32 %0, %8, %14;\n\taddc.cc.u32 %1, %9, %15;\n\taddc.cc.u32 %2, %10, %16;\n\taddc.cc.u32 %3, %11, %17;\n\taddc.cc.u32 %4, %12, %18;\n\taddc.cc.u32 %5, %13, %19;\n\taddc.u32 %6, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(c), "+r"(cin)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]));
        return c;
    }
};

template <>
struct CarryChainIn<7> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[7], const uint32_t (&a)[7],
                                                   const uint32_t (&b)[7], uint32_t cin) {
        uint32_t c;
        asm("add.cc.u32 %8, %8, -1;\n\taddc.cc.u32 %0, %9, %16;\n\taddc.cc.u32 %1, %10, %17;\n\taddc.cc.u32 %2, %11, %18;\n\taddc.cc.u32 %3, %12, %19;\n\taddc.cc.u32 %4, %13, %20;\n\taddc.cc.u32 %5, %14, %21;\n\taddc.cc.u32 %6, %15, %22;\n\taddc.u32 %7, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(c), "+r"(cin)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]));
        return c;
    }
};

template <>
struct CarryChainIn<8> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[8], const uint32_t (&a)[8],
                                                   const uint32_t (&b)[8], uint32_t cin) {
        uint32_t c;
        asm("add.cc.u32 %9, %9, -1;\n\taddc.cc.u32 %0, %10, %18;\n\taddc.cc.u32 %1, %11, %19;\n\taddc.cc.u32 %2, %12, %20;\n\taddc.cc.u32 %3, %13, %21;\n\taddc.cc.u32 %4, %14, %22;\n\taddc.cc.u32 %5, %15, %23;\n\taddc.cc.u32 %6, %16, %24;\n\taddc.cc.u32 %7, %17, %25;\n\taddc.u32 %8, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(s[7]), "=r"(c), "+r"(cin)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
        return c;
    }
};

// The same sum with each word's add issued as a multiply-add by a runtime
// one (madc: s = a * one + b + carry), which can issue on the multiply-add
// pipe instead of the integer ALU pipe; `one` must be 1 and unknown to the
// compiler.
template <int N>
struct CarryChainMadIn;

template <>
struct CarryChainMadIn<1> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[1], const uint32_t (&a)[1],
                                                   const uint32_t (&b)[1], uint32_t cin, uint32_t one) {
        uint32_t c;
        asm("add.cc.u32 %2, %2, -1;\n\tmadc.lo.cc.u32 %0, %3, %5, %4;\n\taddc.u32 %1, 0, 0;"
            : "=r"(s[0]), "=r"(c), "+r"(cin)
            : "r"(a[0]), "r"(b[0]), "r"(one));
        return c;
    }
};

template <>
struct CarryChainMadIn<2> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[2], const uint32_t (&a)[2],
                                                   const uint32_t (&b)[2], uint32_t cin, uint32_t one) {
        uint32_t c;
        asm("add.cc.u32 %3, %3, -1;\n\tmadc.lo.cc.u32 %0, %4, %8, %6;\n\tmadc.lo.cc.u32 %1, %5, %8, %7;\n\taddc.u32 %2, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(c), "+r"(cin)
            : "r"(a[0]), "r"(a[1]), "r"(b[0]), "r"(b[1]), "r"(one));
        return c;
    }
};

template <>
struct CarryChainMadIn<3> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[3], const uint32_t (&a)[3],
                                                   const uint32_t (&b)[3], uint32_t cin, uint32_t one) {
        uint32_t c;
        asm("add.cc.u32 %4, %4, -1;\n\tmadc.lo.cc.u32 %0, %5, %11, %8;\n\tmadc.lo.cc.u32 %1, %6, %11, %9;\n\tmadc.lo.cc.u32 %2, %7, %11, %10;\n\taddc.u32 %3, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(c), "+r"(cin)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(one));
        return c;
    }
};

template <>
struct CarryChainMadIn<4> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[4], const uint32_t (&a)[4],
                                                   const uint32_t (&b)[4], uint32_t cin, uint32_t one) {
        uint32_t c;
        asm("add.cc.u32 %5, %5, -1;\n\tmadc.lo.cc.u32 %0, %6, %14, %10;\n\tmadc.lo.cc.u32 %1, %7, %14, %11;\n\tmadc.lo.cc.u32 %2, %8, %14, %12;\n\tmadc.lo.cc.u32 %3, %9, %14, %13;\n\taddc.u32 %4, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(c), "+r"(cin)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(one));
        return c;
    }
};

template <>
struct CarryChainMadIn<5> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[5], const uint32_t (&a)[5],
                                                   const uint32_t (&b)[5], uint32_t cin, uint32_t one) {
        uint32_t c;
        asm("add.cc.u32 %6, %6, -1;\n\tmadc.lo.cc.u32 %0, %7, %17, %12;\n\tmadc.lo.cc.u32 %1, %8, %17, %13;\n\tmadc.lo.cc.u32 %2, %9, %17, %14;\n\tmadc.lo.cc.u32 %3, %10, %17, %15;\n\tmadc.lo.cc.u32 %4, %11, %17, %16;\n\taddc.u32 %5, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(c), "+r"(cin)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(one));
        return c;
    }
};

template <>
struct CarryChainMadIn<6> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[6], const uint32_t (&a)[6],
                                                   const uint32_t (&b)[6], uint32_t cin, uint32_t one) {
        uint32_t c;
        asm("add.cc.u32 %7, %7, -1;\n\tmadc.lo.cc.u32 %0, %8, %20, %14;\n\tmadc.lo.cc.u32 %1, %9, %20, %15;\n\tmadc.lo.cc.u32 %2, %10, %20, %16;\n\tmadc.lo.cc.u32 %3, %11, %20, %17;\n\tmadc.lo.cc.u32 %4, %12, %20, %18;\n\tmadc.lo.cc.u32 %5, %13, %20, %19;\n\taddc.u32 %6, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(c), "+r"(cin)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(one));
        return c;
    }
};

template <>
struct CarryChainMadIn<7> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[7], const uint32_t (&a)[7],
                                                   const uint32_t (&b)[7], uint32_t cin, uint32_t one) {
        uint32_t c;
        asm("add.cc.u32 %8, %8, -1;\n\tmadc.lo.cc.u32 %0, %9, %23, %16;\n\tmadc.lo.cc.u32 %1, %10, %23, %17;\n\tmadc.lo.cc.u32 %2, %11, %23, %18;\n\tmadc.lo.cc.u32 %3, %12, %23, %19;\n\tmadc.lo.cc.u32 %4, %13, %23, %20;\n\tmadc.lo.cc.u32 %5, %14, %23, %21;\n\tmadc.lo.cc.u32 %6, %15, %23, %22;\n\taddc.u32 %7, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(c), "+r"(cin)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(one));
        return c;
    }
};

template <>
struct CarryChainMadIn<8> {
    static __device__ __forceinline__ uint32_t add(uint32_t (&s)[8], const uint32_t (&a)[8],
                                                   const uint32_t (&b)[8], uint32_t cin, uint32_t one) {
        uint32_t c;
        asm("add.cc.u32 %9, %9, -1;\n\tmadc.lo.cc.u32 %0, %10, %26, %18;\n\tmadc.lo.cc.u32 %1, %11, %26, %19;\n\tmadc.lo.cc.u32 %2, %12, %26, %20;\n\tmadc.lo.cc.u32 %3, %13, %26, %21;\n\tmadc.lo.cc.u32 %4, %14, %26, %22;\n\tmadc.lo.cc.u32 %5, %15, %26, %23;\n\tmadc.lo.cc.u32 %6, %16, %26, %24;\n\tmadc.lo.cc.u32 %7, %17, %26, %25;\n\taddc.u32 %8, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(s[7]), "=r"(c), "+r"(cin)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(one));
        return c;
    }
};

}  // namespace msa
