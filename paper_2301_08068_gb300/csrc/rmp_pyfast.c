/* rmp_pyfast.c -- CPython entry points for the synchronous calls of include/rmp.h
 * (rmp_raycast_eval, rmp_scan_eval): argument marshalling only.  The ctypes binding
 * spends several microseconds per call building ctypes arrays and structures; these
 * functions read x and xdot straight from any object with a float64 buffer (or a
 * sequence of three numbers), call the C function with the GIL released, and return
 * (status, the 144 result bytes).  Handles and pointers arrive as Python ints (the
 * values the ctypes binding already holds). */
#define PY_SSIZE_T_CLEAN
#include <Python.h>
#include <string.h>

#include "rmp.h"

/* Three doubles from a contiguous float64 buffer of 3 items, else from a sequence. */
static int read3(PyObject* o, double v[3]) {
  if (PyObject_CheckBuffer(o)) {
    Py_buffer b;
    if (PyObject_GetBuffer(o, &b, PyBUF_C_CONTIGUOUS | PyBUF_FORMAT) == 0) {
      const int ok = b.len == 3 * (Py_ssize_t)sizeof(double) && b.itemsize == sizeof(double) &&
                     b.format != NULL && (strcmp(b.format, "d") == 0 || strcmp(b.format, "<d") == 0);
      if (ok) memcpy(v, b.buf, 3 * sizeof(double));
      PyBuffer_Release(&b);
      if (ok) return 0;
    } else {
      PyErr_Clear();
    }
  }
  PyObject* seq = PySequence_Fast(o, "x and xdot must hold three numbers");
  if (!seq) return -1;
  if (PySequence_Fast_GET_SIZE(seq) != 3) {
    Py_DECREF(seq);
    PyErr_SetString(PyExc_ValueError, "x and xdot must hold three numbers");
    return -1;
  }
  for (int i = 0; i < 3; ++i) {
    v[i] = PyFloat_AsDouble(PySequence_Fast_GET_ITEM(seq, i));
    if (v[i] == -1.0 && PyErr_Occurred()) {
      Py_DECREF(seq);
      return -1;
    }
  }
  Py_DECREF(seq);
  return 0;
}

static void* as_ptr(PyObject* o) {
  if (o == Py_None) return NULL;
  return PyLong_AsVoidPtr(o);
}

/* raycast_eval(ctx, map_id, x, xdot, n_rays, params_addr, stream, hits_addr, per_ray_addr)
 *   -> (status, bytes) */
static PyObject* py_raycast_eval(PyObject* self, PyObject* args) {
  (void)self;
  PyObject *ctx_o, *x_o, *v_o, *params_o, *stream_o, *hits_o, *per_o;
  unsigned int map_id, n_rays;
  if (!PyArg_ParseTuple(args, "OIOOIOOOO", &ctx_o, &map_id, &x_o, &v_o, &n_rays, &params_o,
                        &stream_o, &hits_o, &per_o))
    return NULL;
  double x[3], xd[3];
  if (read3(x_o, x) || read3(v_o, xd)) return NULL;
  rmp_ctx* ctx = (rmp_ctx*)as_ptr(ctx_o);
  const rmp_params_t* params = (const rmp_params_t*)as_ptr(params_o);
  rmp_stream_t stream = (rmp_stream_t)as_ptr(stream_o);
  rmp_ray_hit_t* hits = (rmp_ray_hit_t*)as_ptr(hits_o);
  float* per = (float*)as_ptr(per_o);
  if (PyErr_Occurred()) return NULL;
  rmp_result_t out;
  memset(&out, 0, sizeof(out));
  int st;
  Py_BEGIN_ALLOW_THREADS
  st = rmp_raycast_eval(ctx, map_id, x, xd, n_rays, params, stream, &out, hits, per);
  Py_END_ALLOW_THREADS
  return Py_BuildValue("(iy#)", st, (const char*)&out, (Py_ssize_t)sizeof(out));
}

/* scan_eval(ctx, points_addr, n, x, xdot, params_addr, stream, per_ray_addr)
 *   -> (status, bytes) */
static PyObject* py_scan_eval(PyObject* self, PyObject* args) {
  (void)self;
  PyObject *ctx_o, *pts_o, *x_o, *v_o, *params_o, *stream_o, *per_o;
  unsigned int n;
  if (!PyArg_ParseTuple(args, "OOIOOOOO", &ctx_o, &pts_o, &n, &x_o, &v_o, &params_o, &stream_o,
                        &per_o))
    return NULL;
  double x[3], xd[3];
  if (read3(x_o, x) || read3(v_o, xd)) return NULL;
  rmp_ctx* ctx = (rmp_ctx*)as_ptr(ctx_o);
  const float* pts = (const float*)as_ptr(pts_o);
  const rmp_params_t* params = (const rmp_params_t*)as_ptr(params_o);
  rmp_stream_t stream = (rmp_stream_t)as_ptr(stream_o);
  float* per = (float*)as_ptr(per_o);
  if (PyErr_Occurred()) return NULL;
  rmp_result_t out;
  memset(&out, 0, sizeof(out));
  int st;
  Py_BEGIN_ALLOW_THREADS
  st = rmp_scan_eval(ctx, pts, n, x, xd, params, stream, &out, per);
  Py_END_ALLOW_THREADS
  return Py_BuildValue("(iy#)", st, (const char*)&out, (Py_ssize_t)sizeof(out));
}

static PyMethodDef kMethods[] = {
    {"raycast_eval", py_raycast_eval, METH_VARARGS,
     "rmp_raycast_eval(ctx, map_id, x, xdot, n_rays, params, stream, hits, per_ray) -> "
     "(status, result bytes)"},
    {"scan_eval", py_scan_eval, METH_VARARGS,
     "rmp_scan_eval(ctx, points, n, x, xdot, params, stream, per_ray) -> (status, result bytes)"},
    {NULL, NULL, 0, NULL}};

static struct PyModuleDef kModule = {PyModuleDef_HEAD_INIT, "_rmp_fast",
                                     "CPython marshalling of the synchronous rmp calls", -1,
                                     kMethods, NULL, NULL, NULL, NULL};

PyMODINIT_FUNC PyInit__rmp_fast(void) { return PyModule_Create(&kModule); }
