// Host stand-in for the CUDA runtime header, enough for the library's
// internal headers and the graph builder's launcher to compile on the host
// in the kernel emulation tests.
#pragma once
typedef void *cudaStream_t;
typedef int cudaError_t;
#define cudaSuccess 0
inline cudaError_t cudaGetLastError() { return cudaSuccess; }
enum cudaFuncAttribute { cudaFuncAttributeMaxDynamicSharedMemorySize = 8 };
template <class T> inline cudaError_t cudaFuncSetAttribute(T, cudaFuncAttribute, int) { return cudaSuccess; }
