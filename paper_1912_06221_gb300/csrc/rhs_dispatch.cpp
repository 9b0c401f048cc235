// Dispatch of the per-order kernel objects by order and precision.
#include "internal.h"

namespace rdg {

#define RDG_DECL(tag, T, n)                                                     \
  int upload_tab_##tag##n();                                                    \
  int launch_edge_##tag##n(const EdgeArgs<T>& a, cudaStream_t s);               \
  int launch_elem_##tag##n(int mode, const ElemArgs<T>& a, cudaStream_t s);     \
  int launch_edge_vol_##tag##n(const EdgeArgs<T>& a, cudaStream_t s);           \
  int launch_elem_lite_##tag##n(int mode, const ElemArgs<T>& a, cudaStream_t s); \
  int launch_fused_##tag##n(int mode, const EdgeArgs<T>& ea, const ElemArgs<T>& a, cudaStream_t s); \
  int launch_edge_only_##tag##n(const EdgeArgs<T>& a, cudaStream_t s);
#define RDG_DECL_ALL(tag, T) \
  RDG_DECL(tag, T, 1) RDG_DECL(tag, T, 2) RDG_DECL(tag, T, 3) RDG_DECL(tag, T, 4) RDG_DECL(tag, T, 5) RDG_DECL(tag, T, 6)
RDG_DECL_ALL(f, float)
RDG_DECL_ALL(d, double)

#define RDG_SWITCH(expr_tag, call)                 \
  switch (N) {                                     \
    case 1: return call(expr_tag, 1);              \
    case 2: return call(expr_tag, 2);              \
    case 3: return call(expr_tag, 3);              \
    case 4: return call(expr_tag, 4);              \
    case 5: return call(expr_tag, 5);              \
    case 6: return call(expr_tag, 6);              \
  }                                                \
  return RDG_EINVAL;

#define CALL_EDGE(tag, n) launch_edge_##tag##n(a, s)
#define CALL_ELEM(tag, n) launch_elem_##tag##n(mode, a, s)
#define CALL_EDGE_VOL(tag, n) launch_edge_vol_##tag##n(a, s)
#define CALL_ELEM_LITE(tag, n) launch_elem_lite_##tag##n(mode, a, s)
#define CALL_FUSED(tag, n) launch_fused_##tag##n(mode, ea, a, s)
#define CALL_EDGE_ONLY(tag, n) launch_edge_only_##tag##n(a, s)

int launch_edge32(int N, const EdgeArgs<float>& a, cudaStream_t s) { RDG_SWITCH(f, CALL_EDGE) }
int launch_edge64(int N, const EdgeArgs<double>& a, cudaStream_t s) { RDG_SWITCH(d, CALL_EDGE) }
int launch_elem32(int N, int mode, const ElemArgs<float>& a, cudaStream_t s) { RDG_SWITCH(f, CALL_ELEM) }
int launch_elem64(int N, int mode, const ElemArgs<double>& a, cudaStream_t s) { RDG_SWITCH(d, CALL_ELEM) }
int launch_edge_vol32(int N, const EdgeArgs<float>& a, cudaStream_t s) { RDG_SWITCH(f, CALL_EDGE_VOL) }
int launch_edge_vol64(int N, const EdgeArgs<double>& a, cudaStream_t s) { RDG_SWITCH(d, CALL_EDGE_VOL) }
int launch_elem_lite32(int N, int mode, const ElemArgs<float>& a, cudaStream_t s) { RDG_SWITCH(f, CALL_ELEM_LITE) }
int launch_elem_lite64(int N, int mode, const ElemArgs<double>& a, cudaStream_t s) { RDG_SWITCH(d, CALL_ELEM_LITE) }
int launch_edge_only32(int N, const EdgeArgs<float>& a, cudaStream_t s) { RDG_SWITCH(f, CALL_EDGE_ONLY) }
int launch_edge_only64(int N, const EdgeArgs<double>& a, cudaStream_t s) { RDG_SWITCH(d, CALL_EDGE_ONLY) }
int launch_fused32(int N, int mode, const EdgeArgs<float>& ea, const ElemArgs<float>& a, cudaStream_t s) {
  RDG_SWITCH(f, CALL_FUSED)
}
int launch_fused64(int N, int mode, const EdgeArgs<double>& ea, const ElemArgs<double>& a, cudaStream_t s) {
  RDG_SWITCH(d, CALL_FUSED)
}

int launch_gemm_f1(const EdgeArgs<float>& a, cudaStream_t s);
int launch_gemm_f2(const EdgeArgs<float>& a, cudaStream_t s);
int launch_gemm_f3(const EdgeArgs<float>& a, cudaStream_t s);
int launch_gemm_f4(const EdgeArgs<float>& a, cudaStream_t s);
int launch_gemm_f5(const EdgeArgs<float>& a, cudaStream_t s);

int launch_gemm32(int N, const EdgeArgs<float>& a, cudaStream_t s) {
  switch (N) {
    case 1: return launch_gemm_f1(a, s);
    case 2: return launch_gemm_f2(a, s);
    case 3: return launch_gemm_f3(a, s);
    case 4: return launch_gemm_f4(a, s);
    case 5: return launch_gemm_f5(a, s);
  }
  return RDG_EINVAL;
}

int launch_volume_f6(const EdgeArgs<float>& a, cudaStream_t s);

bool split_volume32(int N) { return N == 6; }
int launch_volume32(int N, const EdgeArgs<float>& a, cudaStream_t s) {
  return N == 6 ? launch_volume_f6(a, s) : RDG_EINVAL;
}

int gemm_param_words(int N) { return (2 * np_of(N) + nfp_of(N) + 3 + 3) / 4; }

int upload_elem_tables(int device) {
  (void)device;
  int (*fns[])() = {upload_tab_f1, upload_tab_f2, upload_tab_f3, upload_tab_f4, upload_tab_f5, upload_tab_f6,
                    upload_tab_d1, upload_tab_d2, upload_tab_d3, upload_tab_d4, upload_tab_d5, upload_tab_d6};
  for (auto f : fns) {
    int rc = f();
    if (rc != RDG_OK) return rc;
  }
  return RDG_OK;
}

}  // namespace rdg
