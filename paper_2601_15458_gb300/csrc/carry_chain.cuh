// Multi-word additions on the hardware carry chain: one add per 32-bit word
// (word 0 lowest).  A carry flag cannot live across separate asm statements,
// so each word count has its own specialisation written as one statement.
#pragma once

#include <stdint.h>

namespace msa {

// add(s, a, b, cin): s = a + b + cin over N words on the carry chain,
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

}  // namespace msa
