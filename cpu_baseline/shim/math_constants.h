// Host stand-in for the one CUDA math constant the binary64 solid code uses.
#pragma once
#define CUDART_INF (__builtin_inf())
