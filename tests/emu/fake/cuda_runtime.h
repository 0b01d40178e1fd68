// Host stand-in for the CUDA runtime header, enough for the library's
// internal headers to compile on the host in the kernel emulation tests.
#pragma once
typedef void *cudaStream_t;
typedef int cudaError_t;
#define cudaSuccess 0
