// The compile-time specialisations of the FFT passes (tfft_spec.cu,
// tfft_spec_real.cu).
#pragma once

// The table of specialisations: length; contiguous passes: elements per
// thread and lines per CTA; strided passes: elements per thread and tile
// width; radices.  "Elements per thread" is L / (threads per line); for the
// lengths with 2, 3 and 5 all present no radix set divides it, and the
// threads carry ceil(butterflies / threads) butterflies per stage (nbf()).
#define TFFT_SPECS(X)                       \
  X(32, 8, 64, 8, 32, 8, 4)                 \
  X(64, 8, 32, 8, 32, 8, 8)                 \
  X(96, 12, 32, 12, 32, 4, 4, 3, 2)         \
  X(128, 16, 32, 16, 32, 16, 8)             \
  X(160, 20, 32, 20, 32, 5, 4, 4, 2)        \
  X(256, 16, 16, 16, 32, 16, 16)            \
  X(512, 32, 16, 32, 16, 32, 16)            \
  X(60, 15, 64, 15, 64, 4, 5, 3)            \
  X(120, 15, 32, 15, 32, 8, 5, 3)           \
  X(240, 15, 16, 15, 16, 16, 5, 3)          \
  X(480, 30, 16, 30, 16, 16, 5, 3, 2)       \
  X(48, 12, 64, 12, 64, 4, 4, 3)            \
  X(80, 20, 64, 20, 64, 5, 4, 4)            \
  X(192, 12, 16, 12, 16, 4, 4, 4, 3)        \
  X(320, 20, 16, 20, 16, 5, 4, 4, 4)        \
  X(384, 24, 16, 24, 16, 8, 8, 3, 2)        \
  X(640, 20, 8, 20, 8, 5, 4, 4, 4, 2)       \
  X(768, 24, 8, 24, 8, 8, 8, 4, 3)          \
  X(1024, 32, 8, 32, 8, 32, 32)             \
  X(2048, 32, 4, 32, 4, 32, 8, 8)           \
  X(4096, 16, 1, 16, 2, 16, 16, 16)

// Strided passes that use other elements per thread, tile width or radices
// than the row above for the same length: length; elements per thread; tile
// width; radices.  512 with 16 elements (512 threads, 2 CTAs and 32 warps per
// SM) instead of 32 (256 threads, register-limited to 16 warps per SM); 256
// in 16-column tiles (256 threads, 4 CTAs per SM) instead of 32 (512 threads,
// 2 CTAs): the same warps per SM in more, independent CTAs.
#define TFFT_SPECS_STRIDED(X) \
  X(512, 16, 16, 8, 8, 8)           \
  X(256, 16, 16, 16, 16)
