/* A minimal NVTX tool for the tests: loaded by the NVTX calls of a process when
 * NVTX_INJECTION64_PATH names this library, it records the name of every range
 * pushed with nvtxRangePushA, one per line, in the file named by
 * NVTX_RECORD_FILE.  Only the core module's RangePushA / RangePop are hooked. */
#include <stdio.h>
#include <stdlib.h>
#include <nvtx3/nvToolsExt.h>

static FILE *out;

static int record_push(const char *name) {
  if (out && name) {
    fprintf(out, "%s\n", name);
    fflush(out);
  }
  return 0;
}

static int record_pop(void) { return 0; }

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
  const NvtxExportTableCallbacks *cb = (const NvtxExportTableCallbacks *)get_table(NVTX_ETID_CALLBACKS);
  NvtxFunctionTable table = 0;
  unsigned int size = 0;
  const char *path = getenv("NVTX_RECORD_FILE");
  if (!cb || !path || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size)) return 0;
  if (size <= NVTX_CBID_CORE_RangePop) return 0;
  out = fopen(path, "w");
  if (!out) return 0;
  *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)record_push;
  *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)record_pop;
  return 1;
}
