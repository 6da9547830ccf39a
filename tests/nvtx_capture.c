/* A minimal NVTX tool for the tests: loaded through NVTX_INJECTION64_PATH,
 * it records the names of the ranges pushed by the process (the NVTX
 * injection interface of the public nvtx3 headers). */
#include <string.h>

#include <nvtx3/nvToolsExt.h>

static char g_names[8192];
static size_t g_used;
static int g_depth;

static int NVTX_API capture_push(const char *msg)
{
    const size_t n = msg ? strlen(msg) : 0;
    if (g_used + n + 2 < sizeof g_names) {
        memcpy(g_names + g_used, msg, n);
        g_used += n;
        g_names[g_used++] = '\n';
        g_names[g_used] = 0;
    }
    return g_depth++;
}

static int NVTX_API capture_pop(void) { return --g_depth; }

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get)
{
    const NvtxExportTableCallbacks *cb =
        (const NvtxExportTableCallbacks *)get(NVTX_ETID_CALLBACKS);
    NvtxFunctionTable table = 0;
    unsigned int size = 0;
    if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size))
        return 0;
    if (size > NVTX_CBID_CORE_RangePushA)
        *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)capture_push;
    if (size > NVTX_CBID_CORE_RangePop)
        *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)capture_pop;
    return 1;
}

const char *nvtx_capture_names(void) { return g_names; }
int nvtx_capture_depth(void) { return g_depth; }
