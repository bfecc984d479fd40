/* NVTX injection library for tests/test_gpu_nvtx.py (built there with
 * gcc -shared -fPIC).  Loaded through NVTX_INJECTION64_PATH, it takes over
 * the range push and pop entries of NVTX's core callback table and appends
 * one line per call ("push <message>" or "pop") to the file named by
 * KK_NVTX_LOG.  Uses only NVTX's documented tool interface: the export table
 * of callbacks (id 1), the core module (1), and its RangePushA (9) and
 * RangePop (11) slots. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

typedef void (*fn_ptr)(void);
typedef fn_ptr **fn_table;
typedef struct {
  size_t struct_size;
  int (*GetModuleFunctionTable)(int module, fn_table *out_table, unsigned int *out_size);
} callbacks_t;
typedef const void *(*get_export_table_t)(uint32_t id);

enum { ETID_CALLBACKS = 1, CB_MODULE_CORE = 1, CBID_RANGE_PUSH_A = 9, CBID_RANGE_POP = 11 };

static FILE *g_log;

static int push_a(const char *msg) {
  if (g_log) {
    fprintf(g_log, "push %s\n", msg ? msg : "");
    fflush(g_log);
  }
  return 0;
}

static int pop(void) {
  if (g_log) {
    fputs("pop\n", g_log);
    fflush(g_log);
  }
  return 0;
}

int InitializeInjectionNvtx2(get_export_table_t get) {
  const char *path = getenv("KK_NVTX_LOG");
  if (!path || !get) return 0;
  if (!g_log) g_log = fopen(path, "a");
  if (!g_log) return 0;
  const callbacks_t *cb = (const callbacks_t *)get(ETID_CALLBACKS);
  if (!cb || !cb->GetModuleFunctionTable) return 0;
  fn_table table = 0;
  unsigned int size = 0;
  if (!cb->GetModuleFunctionTable(CB_MODULE_CORE, &table, &size) || !table || size < CBID_RANGE_POP) return 0;
  *table[CBID_RANGE_PUSH_A] = (fn_ptr)push_a;
  *table[CBID_RANGE_POP] = (fn_ptr)pop;
  return 1;
}
